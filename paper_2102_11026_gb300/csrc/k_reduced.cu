// Reduced-system kernels: row reductions of the output layer (J^T M J,
// J^T M dJ, J^T a), warp-per-tet cubature (Sec. 5), W_L^T a, the complex-step
// reverse pass (Sec. 4.4) and the FP64 assembly / LU / Newton control.
#include "dae_internal.h"
#include "epilogue.cuh"
#include <algorithm>

namespace dae {

// ------------------------------------------------------- row reductions --
// Per block of 128 output rows n (lumped mass m_n on each DOF, Sec. 3.1):
//   y_n = sum_j J_nj z_j + H[Delta,Delta]_n,  a_n = m_n y_n - dt^2 f_ext,n
//   phi_i += J_ni a_n,  Mr_ij += m_n J_ni J_nj (i <= j),  B_ij += m_n J_ni dJ_nj
// Partial layout per block: [phi (r) | Mr upper (r(r+1)/2, row-major i<=j) | B (r*r, i*r+j)].
constexpr int RR_ROWS = 128;

__global__ void __launch_bounds__(256) k_row_reduce(RowArgs A) {
    if (A.ns && A.ns->done) return;
    __shared__ float Js[kMaxR][RR_ROWS + 1];
    __shared__ float dJs[kMaxR][RR_ROWS + 1];
    __shared__ float ms[RR_ROWS], as[RR_ROWS];
    const int r = A.r, t = threadIdx.x;
    const int n0 = blockIdx.x * RR_ROWS;
    if (t < RR_ROWS) {
        const int n = n0 + t;
        float m = 0.f, a = 0.f;
        if (n < A.N) {
            m = A.mdof[n];
            float y = A.HDD[n];
            for (int j = 0; j < r; ++j) {
                float Jv = A.J[(size_t)j * A.N + n];
                Js[j][t] = Jv;
                dJs[j][t] = A.dJ[(size_t)j * A.N + n];
                y = fmaf(Jv, A.zvec[j], y);
            }
            a = (float)((double)m * y - A.dt * A.dt * (A.f_ext ? (double)A.f_ext[n] : 0.0));
            A.a[n] = a;
        } else {
            for (int j = 0; j < r; ++j) { Js[j][t] = 0.f; dJs[j][t] = 0.f; }
        }
        ms[t] = m;
        as[t] = a;
    }
    __syncthreads();
    const int nsym = r * (r + 1) / 2;
    const int n_ent = r + nsym + r * r;
    float* out = A.part + (size_t)blockIdx.x * A.stride;
    for (int e = t; e < n_ent; e += blockDim.x) {
        float acc = 0.f;
        if (e < r) {
            for (int k = 0; k < RR_ROWS; ++k) acc = fmaf(Js[e][k], as[k], acc);
        } else if (e < r + nsym) {
            int p = e - r, i = 0;
            while (p >= r - i) { p -= r - i; ++i; }
            int j = i + p;
            for (int k = 0; k < RR_ROWS; ++k) acc = fmaf(ms[k] * Js[i][k], Js[j][k], acc);
        } else {
            int p = e - r - nsym, i = p / r, j = p % r;
            for (int k = 0; k < RR_ROWS; ++k) acc = fmaf(ms[k] * Js[i][k], dJs[j][k], acc);
        }
        out[e] = acc;
    }
}

void launch_row_reduce(cudaStream_t s, const RowArgs& a, int n_blocks) {
    k_row_reduce<<<n_blocks, 256, 0, s>>>(a);
}

// ------------------------------------------------------------- cubature --
// Cubature forces and stiffness (Sec. 5) over the sampled tets e in C, with the
// displacement gradient G = dU Dm^{-1} of each tet (F = I + G, formed from nodal
// displacement differences so that small strains keep their accuracy):
//   StVK: E = (G + G^T + G^T G)/2, S = 2 mu E + lam tr(E) I, P = F S,
//         Psi = mu tr(E^2) + lam/2 tr(E)^2
//   NH:   P = mu (F - F^{-T}) + lam ln(J) F^{-T},
//         Psi = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2
//   f_e = V_e P Dm^{-T} (nodes 1..3; node 0 = minus their sum)
// and, for every column j of J on the tet's 12 DOFs, the displacement direction dG_j
// and stress differential dP_j = dP[dG_j]:
//   g_j  = V_e P : dG_j            (= (J_e^T f_e)_j)
//   K_ij = V_e dG_i : dP_j         (= (J_e^T K_e J_e)_ij)
// Work split (the per-tet algebra on every lane, the warp on the r columns):
//   phase A   one tet per lane (up to 32 tets per warp at a time), FP32 in forms free of
//             cancellation (below): F, P, the material terms dP needs, f_e (written out
//             for W_L^T a), the energy (summed in FP64)
//   phase B   per tet, lane j forms dG_j, dP_j and g_j; then the warp adds
//             w_e V_e dG^T dP to a 32 x 32 register-blocked tile (lane: 4 rows x 8
//             columns, the rows and columns broadcast from shared memory as float4)
// Each block sums its warps' tiles and writes one partial row [g (r) | K upper
// (r(r+1)/2, row-major i <= j)] and one FP64 energy: the column sums then add
// n_parts rows instead of one per tet.  Fixed tet-to-warp assignment and summation
// order: bitwise reproducible.
// Cancellation-free forms (all terms at the scale of the result):
//   NH   J - 1 = x = tr G + m2(G) + det G (m2: sum of the principal 2x2 minors),
//        ln J = log1p(x), F - F^{-T} = G + F^{-T} G^T,
//        Psi = mu [(x - log1p x) + 1/2 sum_{i<j} (G_ij + G_ji)^2 + sum_i G_ii^2
//                  - 1/2 (tr G)^2 - det G] + lam/2 (log1p x)^2
//        (the first-order parts of 1/2 (tr F^T F - 3) = tr G + |G|^2/2 and ln J cancel
//        exactly and are left out)
// J columns come from the compact cubature rows when the output stage wrote them
// (Jc: [1 + rq][ldc], row 12 slot + 3 a + d = vertex a, axis d of the slot's tet,
// column 0 = u), else from J ([r][N]) and u ([N]) at the DOFs.
constexpr int kCubWarps = 4;   // warps per block

// x - log1p(x) without cancellation: its Taylor series x^2/2 - x^3/3 + ... for
// |x| < 1/4 (terms to x^14: truncation below 1e-9 of the result), the direct form
// beyond (relative error ~ 2 eps / |x| <= 8 eps there).
__device__ __forceinline__ float xm_log1p(float x) {
    if (fabsf(x) < 0.25f) {
        float s = 0.f;
#pragma unroll
        for (int k = 14; k >= 2; --k) s = fmaf(s, x, ((k & 1) ? -1.f : 1.f) / (float)k);
        return s * x * x;
    }
    return x - log1pf(x);
}

struct CubTet {          // per-tet data phase A leaves for phase B (shared memory)
    float F[9], P[9], M[9];   // M: S (StVK) or F^{-T} (NH)
    float Bm[9];
    float c1;                 // NH: mu - lam ln J
    float wV;                 // w_e V_e
    int v[4];
    int slot;                 // cubature slot; -1: skipped (inverted or invalid)
};

__device__ __forceinline__ void cubature_impl(const CubArgs& A) {
    if (A.ns && A.ns->done) return;
    const int b = blockIdx.x;
    if (b >= A.n_parts) return;
    // the tet records of phase A and, once every warp is done, the warps' tiles
    union Shared { CubTet T[kCubWarps][32]; float K[kCubWarps][32][33]; };
    __shared__ Shared sh;
    auto& sT = sh.T;
    auto& sK = sh.K;
    __shared__ __align__(16) float sdG[kCubWarps][9][32];   // [k][i]: dG_i[k]
    __shared__ __align__(16) float sdP[kCubWarps][9][32];   // [k][j]: w V dP_j[k]
    __shared__ float sg[kCubWarps][32];
    __shared__ double sE[kCubWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = A.r, np = A.np;
    const int nsym = r * (r + 1) / 2;
    const float mu = A.mu, lam = A.lam;
    const float* __restrict__ wts = A.cub_w + (A.ns ? (size_t)A.ns->frame * A.w_stride : 0);
    // this block's slots [s0, s1); warp w takes s0 + w, s0 + w + kCubWarps, ...
    const int s0 = (int)((long long)A.n_cub * b / A.n_parts);
    const int s1 = (int)((long long)A.n_cub * (b + 1) / A.n_parts);
    const int mine = s1 - s0 > warp ? (s1 - s0 - warp + kCubWarps - 1) / kCubWarps : 0;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    float g_acc = 0.f;
    double e_acc = 0.0;
    const int ib = lane >> 2, jb = lane & 3;   // tile block: rows 4 ib.., columns 8 jb..
    for (int t0 = 0; t0 < mine; t0 += 32) {
        const int nb = min(32, mine - t0);
        // ---------------- phase A: one tet per lane
        if (lane < nb) {
            const int slot = s0 + warp + (t0 + lane) * kCubWarps;
            CubTet& T = sT[warp][lane];
            const int tet = A.cub_tets[slot];
            T.slot = slot;
            bool skip = false;
            if (tet < 0 || tet >= A.n_tet) {   // device arrays skip the host's index check
                if (A.eval_flag) atomicExch(A.eval_flag, 2);
                skip = true;
            } else {
                int v[4];
                for (int a = 0; a < 4; ++a) v[a] = A.tets[4 * tet + a];
                float Bm[9];
                for (int i = 0; i < 9; ++i) Bm[i] = A.Bm[9 * (size_t)tet + i];
                const float V = A.vol[tet];
                const float wgt = wts[slot];
                float ue[12];
                if (A.Jc) {
                    const float4* uc = reinterpret_cast<const float4*>(A.Jc + 12 * (size_t)slot);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float4 x = uc[q];
                        ue[4 * q] = x.x; ue[4 * q + 1] = x.y; ue[4 * q + 2] = x.z; ue[4 * q + 3] = x.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 12; ++k) ue[k] = A.u[3 * v[k / 3] + k % 3];
                }
                if (np > 0) {   // linear subspace: + (U p) at the tet's DOFs
                    for (int k = 0; k < 12; ++k) {
                        const int dof = 3 * v[k / 3] + k % 3;
                        float s = 0.f;
                        for (int a = 0; a < np; ++a) s = fmaf(A.J[(size_t)a * A.N + dof], A.pv[a], s);
                        ue[k] += s;
                    }
                }
                // G = dU Bm, dU[d][c] = u(v_{c+1}, d) - u(v_0, d)
                float G[9];
                for (int d = 0; d < 3; ++d)
                    for (int j = 0; j < 3; ++j) {
                        float s = 0.f;
                        for (int c = 0; c < 3; ++c) s = fmaf(ue[3 * (c + 1) + d] - ue[d], Bm[c * 3 + j], s);
                        G[d * 3 + j] = s;
                    }
                float F[9], P[9], M[9], c1 = 0.f, psi = 0.f;
                for (int i = 0; i < 9; ++i) F[i] = G[i] + ((i % 4) == 0 ? 1.f : 0.f);
                if (A.material == DAE_STVK) {
                    float E[9];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float gg = 0.f;
                            for (int k = 0; k < 3; ++k) gg = fmaf(G[k * 3 + i], G[k * 3 + j], gg);
                            E[i * 3 + j] = 0.5f * (G[i * 3 + j] + G[j * 3 + i] + gg);
                        }
                    const float trE = E[0] + E[4] + E[8];
                    float trE2 = 0.f;
                    for (int i = 0; i < 9; ++i) trE2 = fmaf(E[i], E[i], trE2);
                    for (int i = 0; i < 9; ++i) M[i] = 2.f * mu * E[i] + ((i % 4) == 0 ? lam * trE : 0.f);
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float s = 0.f;
                            for (int k = 0; k < 3; ++k) s = fmaf(F[i * 3 + k], M[k * 3 + j], s);
                            P[i * 3 + j] = s;
                        }
                    psi = mu * trE2 + 0.5f * lam * trE * trE;
                } else {
                    const float trG = G[0] + G[4] + G[8];
                    const float m2 = (G[0] * G[4] - G[1] * G[3]) + (G[0] * G[8] - G[2] * G[6]) +
                                     (G[4] * G[8] - G[5] * G[7]);
                    const float d3 = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                                     G[2] * (G[3] * G[7] - G[4] * G[6]);
                    const float x = trG + m2 + d3;   // J - 1
                    if (!(x > -1.f)) {
                        if (A.eval_flag) atomicExch(A.eval_flag, 1);
                        skip = true;
                    } else {
                        const float Jd = 1.f + x, lnJ = log1pf(x), iJ = 1.f / Jd;
                        // F^{-T} = cof(F) / J
                        M[0] = (F[4] * F[8] - F[5] * F[7]) * iJ;
                        M[1] = (F[5] * F[6] - F[3] * F[8]) * iJ;
                        M[2] = (F[3] * F[7] - F[4] * F[6]) * iJ;
                        M[3] = (F[2] * F[7] - F[1] * F[8]) * iJ;
                        M[4] = (F[0] * F[8] - F[2] * F[6]) * iJ;
                        M[5] = (F[1] * F[6] - F[0] * F[7]) * iJ;
                        M[6] = (F[1] * F[5] - F[2] * F[4]) * iJ;
                        M[7] = (F[2] * F[3] - F[0] * F[5]) * iJ;
                        M[8] = (F[0] * F[4] - F[1] * F[3]) * iJ;
                        // P = mu (G + F^{-T} G^T) + lam ln J F^{-T}
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) {
                                float s = 0.f;
                                for (int k = 0; k < 3; ++k) s = fmaf(M[i * 3 + k], G[j * 3 + k], s);
                                P[i * 3 + j] = mu * (G[i * 3 + j] + s) + lam * lnJ * M[i * 3 + j];
                            }
                        c1 = mu - lam * lnJ;
                        float sym = 0.f;
                        sym += (G[1] + G[3]) * (G[1] + G[3]);
                        sym += (G[2] + G[6]) * (G[2] + G[6]);
                        sym += (G[5] + G[7]) * (G[5] + G[7]);
                        const float dia = G[0] * G[0] + G[4] * G[4] + G[8] * G[8];
                        psi = mu * (xm_log1p(x) + 0.5f * sym + dia - 0.5f * trG * trG - d3) +
                              0.5f * lam * lnJ * lnJ;
                    }
                }
                if (!skip) {
                    // nodal forces: H = V P Bm^T, f(node c+1, d) = H[d][c], f(node 0) = -sum
                    float fe[12];
                    for (int d = 0; d < 3; ++d) {
                        float f0 = 0.f;
                        for (int c = 0; c < 3; ++c) {
                            float h = 0.f;
                            for (int k = 0; k < 3; ++k) h = fmaf(P[d * 3 + k], Bm[c * 3 + k], h);
                            h *= V;
                            fe[3 * (c + 1) + d] = wgt * h;
                            f0 -= h;
                        }
                        fe[d] = wgt * f0;
                    }
                    float4* fw = reinterpret_cast<float4*>(A.fe_w + 12 * (size_t)slot);
                    int4* fd = reinterpret_cast<int4*>(A.fe_dof + 12 * (size_t)slot);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        fw[q] = make_float4(fe[4 * q], fe[4 * q + 1], fe[4 * q + 2], fe[4 * q + 3]);
                        int dd[4];
                        for (int u = 0; u < 4; ++u) { const int k = 4 * q + u; dd[u] = 3 * v[k / 3] + k % 3; }
                        fd[q] = make_int4(dd[0], dd[1], dd[2], dd[3]);
                    }
                    e_acc += (double)wgt * (double)V * (double)psi;
                    for (int i = 0; i < 9; ++i) { T.F[i] = F[i]; T.P[i] = P[i]; T.M[i] = M[i]; T.Bm[i] = Bm[i]; }
                    for (int a = 0; a < 4; ++a) T.v[a] = v[a];
                    T.c1 = c1;
                    T.wV = wgt * V;
                }
            }
            if (skip) {
                T.slot = -1;
                float4* fw = reinterpret_cast<float4*>(A.fe_w + 12 * (size_t)slot);
                int4* fd = reinterpret_cast<int4*>(A.fe_dof + 12 * (size_t)slot);
                for (int q = 0; q < 3; ++q) { fw[q] = make_float4(0.f, 0.f, 0.f, 0.f); fd[q] = make_int4(0, 0, 0, 0); }
            }
        }
        __syncwarp();
        // ---------------- phase B: the warp on the tet's r columns
        for (int e = 0; e < nb; ++e) {
            const CubTet& T = sT[warp][e];
            if (T.slot < 0) continue;   // uniform over the warp
            float dG[9], dP[9];
            if (lane < r) {
                float Jg[12];
                if (A.Jc && lane >= np) {
                    const float4* jc = reinterpret_cast<const float4*>(
                        A.Jc + (size_t)(1 + lane - np) * A.ldc + 12 * (size_t)T.slot);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float4 x = jc[q];
                        Jg[4 * q] = x.x; Jg[4 * q + 1] = x.y; Jg[4 * q + 2] = x.z; Jg[4 * q + 3] = x.w;
                    }
                } else {
                    const float* Jcol = A.J + (size_t)lane * A.N;
#pragma unroll
                    for (int k = 0; k < 12; ++k) Jg[k] = Jcol[3 * T.v[k / 3] + k % 3];
                }
                for (int d = 0; d < 3; ++d)
                    for (int j = 0; j < 3; ++j) {
                        float s = 0.f;
                        for (int c = 0; c < 3; ++c) s = fmaf(Jg[3 * (c + 1) + d] - Jg[d], T.Bm[c * 3 + j], s);
                        dG[d * 3 + j] = s;
                    }
                if (A.material == DAE_STVK) {
                    // dE = (dG^T F + F^T dG)/2, dS = 2 mu dE + lam tr(dE) I, dP = dG S + F dS
                    float dE[9];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float s = 0.f;
                            for (int k = 0; k < 3; ++k)
                                s = fmaf(dG[k * 3 + i], T.F[k * 3 + j], fmaf(T.F[k * 3 + i], dG[k * 3 + j], s));
                            dE[i * 3 + j] = 0.5f * s;
                        }
                    const float trdE = dE[0] + dE[4] + dE[8];
                    float dS[9];
                    for (int i = 0; i < 9; ++i) dS[i] = 2.f * mu * dE[i] + ((i % 4) == 0 ? lam * trdE : 0.f);
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float s = 0.f;
                            for (int k = 0; k < 3; ++k)
                                s = fmaf(dG[i * 3 + k], T.M[k * 3 + j], fmaf(T.F[i * 3 + k], dS[k * 3 + j], s));
                            dP[i * 3 + j] = s;
                        }
                } else {
                    // dP = mu dG + (mu - lam lnJ) F^{-T} dG^T F^{-T} + lam (F^{-T}:dG) F^{-T}
                    float tr = 0.f;
                    for (int i = 0; i < 9; ++i) tr = fmaf(T.M[i], dG[i], tr);
                    float M1[9];   // F^{-T} dG^T
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float s = 0.f;
                            for (int k = 0; k < 3; ++k) s = fmaf(T.M[i * 3 + k], dG[j * 3 + k], s);
                            M1[i * 3 + j] = s;
                        }
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            float s = 0.f;
                            for (int k = 0; k < 3; ++k) s = fmaf(M1[i * 3 + k], T.M[k * 3 + j], s);
                            dP[i * 3 + j] = mu * dG[i * 3 + j] + T.c1 * s + lam * tr * T.M[i * 3 + j];
                        }
                }
                float gs = 0.f;
                for (int i = 0; i < 9; ++i) gs = fmaf(T.P[i], dG[i], gs);
                g_acc = fmaf(T.wV, gs, g_acc);
            } else {
                for (int i = 0; i < 9; ++i) { dG[i] = 0.f; dP[i] = 0.f; }
            }
            for (int k = 0; k < 9; ++k) {
                sdG[warp][k][lane] = dG[k];
                sdP[warp][k][lane] = T.wV * dP[k];
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float4 gi = *reinterpret_cast<const float4*>(&sdG[warp][k][4 * ib]);
                const float4 p0 = *reinterpret_cast<const float4*>(&sdP[warp][k][8 * jb]);
                const float4 p1 = *reinterpret_cast<const float4*>(&sdP[warp][k][8 * jb + 4]);
                const float gv[4] = {gi.x, gi.y, gi.z, gi.w};
                const float pv[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(gv[a], pv[c], acc[a][c]);
            }
            __syncwarp();
        }
        __syncwarp();
    }
    // ---------------- block sums: one partial row and one energy per block
    __syncthreads();   // every warp is past phase B: the tet records may be overwritten
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) sK[warp][4 * ib + a][8 * jb + c] = acc[a][c];
    sg[warp][lane] = g_acc;
    for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    if (lane == 0) sE[warp] = e_acc;
    __syncthreads();
    float* part = A.part + (size_t)b * A.stride;
    for (int e = threadIdx.x; e < r + nsym; e += blockDim.x) {
        float s = 0.f;
        if (e < r) {
            for (int w = 0; w < kCubWarps; ++w) s += sg[w][e];
        } else {
            int p = e - r, i = 0;
            while (p >= r - i) { p -= r - i; ++i; }
            const int j = i + p;
            for (int w = 0; w < kCubWarps; ++w) s += sK[w][i][j];
        }
        part[e] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kCubWarps; ++w) s += sE[w];
        A.energy[b] = s;
    }
}

__global__ void __launch_bounds__(32 * kCubWarps) k_cubature(CubArgs A) { cubature_impl(A); }

// Grouped form: z = system.
__global__ void __launch_bounds__(32 * kCubWarps) k_cubature_b(const CubArgs* __restrict__ args) {
    cubature_impl(args[blockIdx.z]);
}

// Partial rows of a cubature set: one block per kCubWarps tets up to 4 blocks per SM.
int cubature_parts(int n_cub, int sm_count) {
    if (n_cub <= 0) return 0;
    return std::max(1, std::min((n_cub + kCubWarps - 1) / kCubWarps, 4 * sm_count));
}

void launch_cubature_batched(cudaStream_t s, const CubArgs* d_args, int n_sys, int max_parts) {
    if (n_sys <= 0 || max_parts <= 0) return;
    k_cubature_b<<<dim3(max_parts, 1, n_sys), 32 * kCubWarps, 0, s>>>(d_args);
}

void launch_cubature(cudaStream_t s, const CubArgs& a) {
    if (a.n_cub <= 0 || a.n_parts <= 0) return;
    k_cubature<<<a.n_parts, 32 * kCubWarps, 0, s>>>(a);
}

// ---------------------------------------------------------- W_L^T a GEMV --
// part[s][k] = sum_{n in split s} W[n][k] a_n                       (s < nsplit_dense)
// part[nsplit_dense + t][k] = dt^2 sum_{p in pair split t} W[dof_p][k] (w f)_p
// (the cubature rows; pairs may repeat a DOF, which only adds).
// Thread = 4 consecutive k (float4), 4 rows in flight.
__device__ __forceinline__ void fma4(float4& acc, const float4& w, float a) {
    acc.x = fmaf(w.x, a, acc.x);
    acc.y = fmaf(w.y, a, acc.y);
    acc.z = fmaf(w.z, a, acc.z);
    acc.w = fmaf(w.w, a, acc.w);
}

__device__ __forceinline__ void wta_impl(const WtaArgs& A) {
    if (skip_reverse(A.ns)) return;
    if (A.run_flag && *A.run_flag == 0) return;
    const int k4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (k4 >= A.K) return;
    const int s = blockIdx.y;
    if (s >= A.nsplit_dense + A.nsplit_pairs + (A.pext ? 1 : 0) + (A.gy ? 1 : 0)) return;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < A.nsplit_dense) {
        const int per = (A.N + A.nsplit_dense - 1) / A.nsplit_dense;
        const int n0 = s * per, n1 = min(A.N, n0 + per);
        int n = n0;
        for (; n + 4 <= n1; n += 4) {
            float4 w[4];
            float av[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = __ldg(reinterpret_cast<const float4*>(A.W + (size_t)(n + u) * A.ld + k4));
                av[u] = __ldg(A.a + n + u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) fma4(acc, w[u], av[u]);
        }
        for (; n < n1; ++n)
            fma4(acc, __ldg(reinterpret_cast<const float4*>(A.W + (size_t)n * A.ld + k4)),
                 __ldg(A.a + n));
    } else if (s < A.nsplit_dense + A.nsplit_pairs) {
        const int t = s - A.nsplit_dense;
        const int per = (A.n_pairs + A.nsplit_pairs - 1) / A.nsplit_pairs;
        const int p0 = t * per, p1 = min(A.n_pairs, p0 + per);
        // FP32 scale (the per-pair FP64 product cost more than the row loads); all of
        // this split's DOFs and weights first, so the row loads issue back to back
        const float dt2 = (float)A.dt2;
        int p = p0;
        for (; p + 8 <= p1; p += 8) {
            int n[8];
            float av[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) { n[u] = __ldg(A.fe_dof + p + u); av[u] = dt2 * __ldg(A.fe_w + p + u); }
            float4 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                w[u] = __ldg(reinterpret_cast<const float4*>(A.Wp + (size_t)n[u] * A.ldp + k4));
#pragma unroll
            for (int u = 0; u < 8; ++u) fma4(acc, w[u], av[u]);
        }
        for (; p < p1; ++p) {
            const int n = A.fe_dof[p];
            const float av = dt2 * A.fe_w[p];
            fma4(acc, __ldg(reinterpret_cast<const float4*>(A.Wp + (size_t)n * A.ldp + k4)), av);
        }
    } else if (A.gy && s == A.nsplit_dense + A.nsplit_pairs + (A.pext ? 1 : 0)) {
        // G x_y from the Gram tiles of the output stage (the dense W_L^T M y)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float v = (k4 + u < A.K) ? A.gy[k4 + u] : 0.f;
            if (u == 0) acc.x = v; else if (u == 1) acc.y = v; else if (u == 2) acc.z = v; else acc.w = v;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float v = (k4 + u < A.K) ? A.pext_scale * A.pext[k4 + u] : 0.f;
            if (u == 0) acc.x = v; else if (u == 1) acc.y = v; else if (u == 2) acc.z = v; else acc.w = v;
        }
    }
    // scalar stores: the partial rows have stride K, which need not keep 16-byte alignment
    float* out = A.part + (size_t)s * A.K + k4;
    const float v[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (k4 + u < A.K) out[u] = v[u];
}

__global__ void __launch_bounds__(256) k_wta(WtaArgs A) { wta_impl(A); }

// Grouped form: z = system.
__global__ void __launch_bounds__(256) k_wta_b(const WtaArgs* __restrict__ args) {
    wta_impl(args[blockIdx.z]);
}

void launch_wta_batched(cudaStream_t s, const WtaArgs* d_args, int n_sys, int max_K, int max_splits) {
    if (n_sys <= 0) return;
    k_wta_b<<<dim3((max_K + 1023) / 1024, max_splits, n_sys), 256, 0, s>>>(d_args);
}

void launch_wta(cudaStream_t s, const WtaArgs& a) {
    dim3 grid((a.K + 1023) / 1024, a.nsplit_dense + a.nsplit_pairs + (a.pext ? 1 : 0) + (a.gy ? 1 : 0));
    k_wta<<<grid, 256, 0, s>>>(a);
}

// x_y[k] = sum_j X[b_j][k] z_j / h + X[g0][k] / h^2 over the output layer's input
// activations (stacked columns, see dae_internal.h), so that J z + H[D,D] = W_L x_y.
__device__ __forceinline__ void xy_impl(const float* X, int ld, int K, int r, const float* zvec,
                                        double h, float* xy, const NewtonState* ns) {
    if (skip_reverse(ns)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float ih = (float)(1.0 / h), ih2 = (float)(1.0 / (h * h));
    float acc = X[(size_t)3 * ld + k] * ih2;
    for (int j = 0; j < r; ++j) acc = fmaf(X[(size_t)(kShared + 3 * j) * ld + k] * ih, zvec[j], acc);
    xy[k] = acc;
}

__global__ void k_xy(const float* X, int ld, int K, int r, const float* zvec, double h, float* xy,
                     const NewtonState* ns) {
    xy_impl(X, ld, K, r, zvec, h, xy, ns);
}

__global__ void k_xy_b(const XyArgs* __restrict__ args) {
    const XyArgs& a = args[blockIdx.z];
    xy_impl(a.X, a.ld, a.K, a.r, a.zvec, a.h, a.xy, a.ns);
}

void launch_xy_batched(cudaStream_t s, const XyArgs* d_args, int n_sys, int max_K) {
    if (n_sys <= 0 || max_K <= 0) return;
    k_xy_b<<<dim3((max_K + 63) / 64, 1, n_sys), 64, 0, s>>>(d_args);
}

void launch_xy(cudaStream_t s, const float* X, int ld, int K, int r, const float* zvec, double h,
               float* xy, const NewtonState* ns) {
    k_xy<<<(K + 63) / 64, 64, 0, s>>>(X, ld, K, r, zvec, h, xy, ns);
}

// out[i][k] = m[i] * W[i][k] for i < rows, k < ld (set-up of G).
__global__ void k_scale_rows(const float* W, int ld, const float* m, int rows, float* out) {
    const size_t n = (size_t)rows * ld;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = W[i] * m[i / ld];
}

void launch_scale_rows(cudaStream_t s, const float* W, int ld, const float* m, int rows, float* out) {
    k_scale_rows<<<1024, 256, 0, s>>>(W, ld, m, rows, out);
}

// flag |= (f != prev) anywhere
__global__ void k_fext_check(const float* f, const float* prev, int N, int* flag) {
    int diff = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        diff |= (__float_as_uint(f[i]) != __float_as_uint(prev[i]));
    diff = __syncthreads_or(diff);
    if (threadIdx.x == 0 && diff) atomicOr(flag, 1);
}

void launch_fext_check(cudaStream_t s, const float* f, const float* prev, int N, int* flag) {
    k_fext_check<<<64, 256, 0, s>>>(f, prev, N, flag);
}

// pext = sum of the split partials; remember f; clear the flag (only when flagged)
__global__ void k_pext_finish(const float* part, int splits, int K, float* pext, const float* f,
                              float* prev, int N, int* flag) {
    if (*flag == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < K) {
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += part[(size_t)s * K + i];
        pext[i] = acc;
    }
    for (int j = i; j < N; j += gridDim.x * blockDim.x) prev[j] = f[j];
}

__global__ void k_clear_flag(int* flag) { *flag = 0; }

void launch_pext_finish(cudaStream_t s, const float* part, int splits, int K, float* pext,
                        const float* f, float* prev, int N, int* flag) {
    k_pext_finish<<<(K + 255) / 256, 256, 0, s>>>(part, splits, K, pext, f, prev, N, flag);
    k_clear_flag<<<1, 1, 0, s>>>(flag);
}

// ------------------------------------------------- complex-step reverse --
// Complex-step backpropagation of g(q) = a . D(q) (Sec. 4.4): the forward pass
// carried q + h e_j i1 for every j; delta has a real column and one i1 column
// per j.  Through the activation of layer l (pre-activation a + b_j i1):
//   Re(g)   = Re(delta) act'(a)
//   Im_j(g) = Im_j(delta) act'(a) + Re(delta) act''(a) b_j
// (terms of relative order h^2 dropped as in the forward pass), then
// delta_{l-1} = W_l^T g.  At the input Re = J^T a and Im_j / h = (a^T H)[:, j].
// Incoming partials [in_split][in_ncol][n_o] are summed in a fixed order.
constexpr int BW_THREADS = 128, BW_CHUNK = 32;

// g[c][k] for k < n_o from the incoming partials (fixed summation order); one
// thread per k forms the real part once and every i1 column from it.
__global__ void k_bwd_prep(BwdArgs A) {
    if (skip_reverse(A.ns)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= A.n_o) return;
    const int r = A.r;
    const size_t stride = (size_t)A.in_ncol * A.n_o;
    float re = 0.f;
    for (int s = 0; s < A.in_split; ++s) re += A.in_part[(size_t)s * stride + k];
    const float s1 = A.S1[k];
    A.g[k] = re * s1;
    for (int c = 1; c <= r; ++c) {
        float im = 0.f;
        if (A.in_ncol > 1)
            for (int s = 0; s < A.in_split; ++s) im += A.in_part[(size_t)s * stride + (size_t)c * A.n_o + k];
        A.g[(size_t)c * A.n_o + k] = fmaf(im, s1, re * A.T[(size_t)(c - 1) * A.n_o + k]);
    }
}

// out_part[s][c][m] = sum_{k in split s} W[k][m] g[c][k]; a thread owns two
// consecutive m (one 8-byte weight load per k), g is staged in shared memory
// and read as float4 over c.
template <int NCOL>
__global__ void __launch_bounds__(BW_THREADS) k_bwd(BwdArgs A) {
    if (skip_reverse(A.ns)) return;
    __shared__ __align__(16) float gs[BW_CHUNK][NCOL];
    const int m = (blockIdx.x * BW_THREADS + threadIdx.x) * 2;
    const int ncol = 1 + A.r;
    const int per = (A.n_o + A.out_split - 1) / A.out_split;
    const int k0 = blockIdx.y * per, k1 = min(A.n_o, k0 + per);
    float acc0[NCOL], acc1[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) { acc0[c] = 0.f; acc1[c] = 0.f; }
    const bool active = m < A.n_i;
    for (int kc = k0; kc < k1; kc += BW_CHUNK) {
        const int kn = min(BW_CHUNK, k1 - kc);
        __syncthreads();
        for (int e = threadIdx.x; e < BW_CHUNK * NCOL; e += BW_THREADS) {
            const int kk = e / NCOL, c = e % NCOL;
            gs[kk][c] = (kk < kn && c < ncol) ? A.g[(size_t)c * A.n_o + kc + kk] : 0.f;
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int kk = 0; kk < kn; ++kk) {
                const float2 w = __ldg(reinterpret_cast<const float2*>(A.W + (size_t)(kc + kk) * A.ld + m));
#pragma unroll
                for (int c4 = 0; c4 < NCOL / 4; ++c4) {
                    const float4 g = *reinterpret_cast<const float4*>(&gs[kk][4 * c4]);
                    acc0[4 * c4 + 0] = fmaf(w.x, g.x, acc0[4 * c4 + 0]);
                    acc0[4 * c4 + 1] = fmaf(w.x, g.y, acc0[4 * c4 + 1]);
                    acc0[4 * c4 + 2] = fmaf(w.x, g.z, acc0[4 * c4 + 2]);
                    acc0[4 * c4 + 3] = fmaf(w.x, g.w, acc0[4 * c4 + 3]);
                    acc1[4 * c4 + 0] = fmaf(w.y, g.x, acc1[4 * c4 + 0]);
                    acc1[4 * c4 + 1] = fmaf(w.y, g.y, acc1[4 * c4 + 1]);
                    acc1[4 * c4 + 2] = fmaf(w.y, g.z, acc1[4 * c4 + 2]);
                    acc1[4 * c4 + 3] = fmaf(w.y, g.w, acc1[4 * c4 + 3]);
                }
            }
        }
    }
    if (active) {
        float* out = A.out_part + (size_t)blockIdx.y * ncol * A.n_i;
#pragma unroll
        for (int c = 0; c < NCOL; ++c) {
            if (c < ncol) {
                out[(size_t)c * A.n_i + m] = acc0[c];
                if (m + 1 < A.n_i) out[(size_t)c * A.n_i + m + 1] = acc1[c];
            }
        }
    }
}

// Tensor-core variant of the top-layer seed: g[c][k] for k < ld (zero padding), c < Cb.
// A block takes 32 consecutive k; its 8 warps sum every 8th incoming split partial
// (coalesced over k), combine the 8 sums in a fixed order, then write the columns
// c = warp, warp + 8, ...
__device__ __forceinline__ void bwd_prep_tc_impl(const BwdArgs& A, int Cb, int ld, float* g32,
                                                 __nv_bfloat16* gh, __nv_bfloat16* gl,
                                                 int out_f32, int out_bf16) {
    if (skip_reverse(A.ns)) return;
    if ((int)blockIdx.x * 32 >= ld) return;
    __shared__ float part[8][kMaxR + 1][33];
    __shared__ float sre[32];
    const int tx = threadIdx.x & 31, sy = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + tx;
    const int r = A.r;
    const size_t stride = (size_t)A.in_ncol * A.n_o;
    const bool valid = k < A.n_o;
    const int ncol = A.in_ncol > 1 ? r + 1 : 1;
    for (int c = 0; c < ncol; ++c) {
        float acc = 0.f;
        if (valid)
            for (int s = sy; s < A.in_split; s += 8) acc += A.in_part[(size_t)s * stride + (size_t)c * A.n_o + k];
        part[sy][c][tx] = acc;
    }
    __syncthreads();
    if (sy == 0) {
        float v = 0.f;
        for (int q = 0; q < 8; ++q) v += part[q][0][tx];
        sre[tx] = v;
    }
    __syncthreads();
    if (k >= ld) return;
    const float re = sre[tx];
    const float s1 = valid ? A.S1[k] : 0.f;
    for (int c = sy; c < Cb; c += 8) {
        float v = 0.f;
        if (valid) {
            if (c == 0) {
                v = re * s1;
            } else if (c <= r) {
                float im = 0.f;
                if (A.in_ncol > 1)
                    for (int q = 0; q < 8; ++q) im += part[q][c][tx];
                v = fmaf(im, s1, re * A.T[(size_t)(c - 1) * A.n_o + k]);
            }
        }
        const size_t idx = (size_t)c * ld + k;
        if (out_f32) g32[idx] = (out_f32 == 2) ? tf32_rna(v) : v;
        if (out_bf16) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            gh[idx] = hi;
            if (out_bf16 == 2) gl[idx] = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
    }
}

__global__ void __launch_bounds__(256) k_bwd_prep_tc(BwdArgs A, int Cb, int ld, float* g32,
                                                     __nv_bfloat16* gh, __nv_bfloat16* gl,
                                                     int out_f32, int out_bf16) {
    bwd_prep_tc_impl(A, Cb, ld, g32, gh, gl, out_f32, out_bf16);
}

__global__ void __launch_bounds__(256) k_bwd_prep_tc_b(const PrepArgs* __restrict__ args) {
    const PrepArgs& p = args[blockIdx.z];
    bwd_prep_tc_impl(p.a, p.Cb, p.ld, p.g32, p.gh, p.gl, p.out_f32, p.out_bf16);
}

void launch_bwd_prep_tc_batched(cudaStream_t s, const PrepArgs* d_args, int n_sys, int max_ld) {
    if (n_sys <= 0) return;
    k_bwd_prep_tc_b<<<dim3((max_ld + 31) / 32, 1, n_sys), 256, 0, s>>>(d_args);
}

void launch_bwd_prep_tc(cudaStream_t s, const BwdArgs& a, int Cb, int ld, float* g32,
                        __nv_bfloat16* gh, __nv_bfloat16* gl, int out_f32, int out_bf16) {
    k_bwd_prep_tc<<<(ld + 31) / 32, 256, 0, s>>>(a, Cb, ld, g32, gh, gl, out_f32, out_bf16);
}

// WT[c][r] = W[r][c] for r < rows, c < cols (zero elsewhere in WT's padding is kept)
__global__ void k_transpose(const float* W, int ld, int rows, int cols, float* WT, int ldT) {
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? W[(size_t)r * ld + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) WT[(size_t)c * ldT + r] = t[threadIdx.x][i];
    }
}

void launch_transpose(cudaStream_t s, const float* W, int ld, int rows, int cols, float* WT, int ldT) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(W, ld, rows, cols, WT, ldT);
}

int bwd_split(int n_i, int n_o, int sm) {
    const int mb = (n_i + 2 * BW_THREADS - 1) / (2 * BW_THREADS);
    return std::max(1, std::min((3 * sm + mb - 1) / mb, std::max(1, n_o / 32)));
}

void launch_bwd(cudaStream_t s, const BwdArgs& a) {
    const int ncol = 1 + a.r;
    k_bwd_prep<<<(a.n_o + 255) / 256, 256, 0, s>>>(a);
    dim3 grid((a.n_i + 2 * BW_THREADS - 1) / (2 * BW_THREADS), a.out_split);
    if (ncol <= 8) k_bwd<8><<<grid, BW_THREADS, 0, s>>>(a);
    else if (ncol <= 16) k_bwd<16><<<grid, BW_THREADS, 0, s>>>(a);
    else if (ncol <= 24) k_bwd<24><<<grid, BW_THREADS, 0, s>>>(a);
    else if (ncol <= 32) k_bwd<32><<<grid, BW_THREADS, 0, s>>>(a);
    else k_bwd<36><<<grid, BW_THREADS, 0, s>>>(a);
}

// ---------------------------------------------------------- weight network --
// Weight prediction (Sec. 5): the first layer over the output layer's input column
// (one warp per row, lanes over K), then the small layers and the squared output rows of
// the cubature tets in one block.
__device__ __forceinline__ bool wnet_skip(const WnetArgs& a) {
    return a.ns && (a.ns->done || (a.first_only && a.ns->evals != 0));
}

// first layer: one block per row, the K products spread over the block's threads
__global__ void __launch_bounds__(256) k_wnet_first(WnetArgs a) {
    if (wnet_skip(a)) return;
    __shared__ float red[8];
    const int i = blockIdx.x;
    const float* __restrict__ row = a.B1 + (size_t)i * a.ldx;
    const float* __restrict__ x = a.x;
    float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    int k = threadIdx.x;
    for (; k + 768 < a.K; k += 1024) {
        acc0 = fmaf(row[k], x[k], acc0);
        acc1 = fmaf(row[k + 256], x[k + 256], acc1);
        acc2 = fmaf(row[k + 512], x[k + 512], acc2);
        acc3 = fmaf(row[k + 768], x[k + 768], acc3);
    }
    for (; k < a.K; k += 256) acc0 = fmaf(row[k], x[k], acc0);
    float acc = (acc0 + acc1) + (acc2 + acc3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        a.h1[i] = sinf(t + a.c1[i]);
    }
}

__device__ __forceinline__ void wnet_layer(const float* __restrict__ A, const float* __restrict__ b,
                                           const float* in, int n_in, float* out, int n_out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < n_out; i += nw) {
        float acc = 0.f;
        for (int k = lane; k < n_in; k += 32) acc = fmaf(A[(size_t)i * n_in + k], in[k], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[i] = sinf(acc + b[i]);
    }
}

// the two small hidden layers (one block); h3 goes to the h1 buffer's tail
__global__ void __launch_bounds__(1024) k_wnet_mid(WnetArgs a) {
    if (wnet_skip(a)) return;
    __shared__ float h1[kMaxWnetWidth], h2[kMaxWnetWidth], h3[kMaxWnetWidth];
    for (int i = threadIdx.x; i < a.H1; i += blockDim.x) h1[i] = a.h1[i];
    __syncthreads();
    wnet_layer(a.A2, a.b2, h1, a.H1, h2, a.H2);
    __syncthreads();
    wnet_layer(a.A3, a.b3, h2, a.H2, h3, a.H3);
    __syncthreads();
    for (int i = threadIdx.x; i < a.H3; i += blockDim.x) a.h1[kMaxWnetWidth + i] = h3[i];
}

// squared output rows of the cubature tets: one warp per tet
__global__ void __launch_bounds__(256) k_wnet_out(WnetArgs a) {
    if (wnet_skip(a)) return;
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= a.n) return;
    const int t = a.tets[j];
    const float* __restrict__ row = a.A4 + (size_t)t * a.H3;
    const float* __restrict__ h3 = a.h1 + kMaxWnetWidth;
    float acc = 0.f;
    for (int k = lane; k < a.H3; k += 32) acc = fmaf(row[k], h3[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const float z = acc + a.b4[t];
        a.w[j] = z * z;
    }
}

// Grouped forms: z = system (systems without a network have H1 = 0 and n = 0).
__global__ void __launch_bounds__(256) k_wnet_first_b(const WnetArgs* __restrict__ args) {
    const WnetArgs& a = args[blockIdx.z];
    if ((int)blockIdx.x >= a.H1) return;
    if (wnet_skip(a)) return;
    __shared__ float red[8];
    const int i = blockIdx.x;
    const float* __restrict__ row = a.B1 + (size_t)i * a.ldx;
    const float* __restrict__ x = a.x;
    float acc = 0.f;
    for (int k = threadIdx.x; k < a.K; k += 256) acc = fmaf(row[k], x[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        a.h1[i] = sinf(t + a.c1[i]);
    }
}

__global__ void __launch_bounds__(1024) k_wnet_mid_b(const WnetArgs* __restrict__ args) {
    const WnetArgs& a = args[blockIdx.z];
    if (a.H1 <= 0 || wnet_skip(a)) return;
    __shared__ float h1[kMaxWnetWidth], h2[kMaxWnetWidth], h3[kMaxWnetWidth];
    for (int i = threadIdx.x; i < a.H1; i += blockDim.x) h1[i] = a.h1[i];
    __syncthreads();
    wnet_layer(a.A2, a.b2, h1, a.H1, h2, a.H2);
    __syncthreads();
    wnet_layer(a.A3, a.b3, h2, a.H2, h3, a.H3);
    __syncthreads();
    for (int i = threadIdx.x; i < a.H3; i += blockDim.x) a.h1[kMaxWnetWidth + i] = h3[i];
}

__global__ void __launch_bounds__(256) k_wnet_out_b(const WnetArgs* __restrict__ args) {
    const WnetArgs& a = args[blockIdx.z];
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= a.n || wnet_skip(a)) return;
    const int t = a.tets[j];
    const float* __restrict__ row = a.A4 + (size_t)t * a.H3;
    const float* __restrict__ h3 = a.h1 + kMaxWnetWidth;
    float acc = 0.f;
    for (int k = lane; k < a.H3; k += 32) acc = fmaf(row[k], h3[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const float z = acc + a.b4[t];
        a.w[j] = z * z;
    }
}

void launch_wnet_batched(cudaStream_t s, const WnetArgs* d_args, int n_sys, int max_H1, int max_n) {
    if (n_sys <= 0 || max_H1 <= 0) return;
    k_wnet_first_b<<<dim3(max_H1, 1, n_sys), 256, 0, s>>>(d_args);
    k_wnet_mid_b<<<dim3(1, 1, n_sys), 1024, 0, s>>>(d_args);
    if (max_n > 0) k_wnet_out_b<<<dim3((max_n + 7) / 8, 1, n_sys), 256, 0, s>>>(d_args);
}

void launch_wnet(cudaStream_t s, const WnetArgs& a) {
    k_wnet_first<<<a.H1, 256, 0, s>>>(a);
    k_wnet_mid<<<1, 1024, 0, s>>>(a);
    if (a.n > 0) k_wnet_out<<<(a.n + 7) / 8, 256, 0, s>>>(a);
}

// ------------------------------------------------------- linear subspace --
// V^T X over 64 rows k per block (the Gram-form analogue of U^T M J, U^T M dJ, U^T M y):
// column c' = 0 -> plane 3 (h^2 H[D,D]), 1 + j -> plane kShared + 3j (h J), 1 + r + j ->
// plane kShared + 3j + 2 (h^3 dJ); scaled by the control.  vz = V z_p per row.
constexpr int kLinRows = 64;
__device__ __forceinline__ void linear_impl(const LinArgs& A) {
    if (A.ns && A.ns->done) return;
    __shared__ float sx[1 + 2 * kMaxR][kLinRows];
    __shared__ float sv[kMaxR][kLinRows];
    __shared__ float szp[kMaxR];
    const int t = threadIdx.x, np = A.np, r = A.r, nc = 1 + 2 * r;
    const double* q = A.q_in ? A.q_in : A.ns->q_trial;
    if (t < np) {
        const double zp = (q[t] - A.qbar[t]) - A.dt * A.qbar_dot[t];
        szp[t] = (float)zp;
        if (blockIdx.x == 0) {
            A.zpv[t] = (float)zp;
            A.zpv[np + t] = (float)q[t];
        }
    }
    const int k = blockIdx.x * kLinRows + t;
    const bool ok = k < A.K;
    for (int cc = 0; cc < nc; ++cc) {
        const int c = cc == 0 ? 3 : (cc <= r ? kShared + 3 * (cc - 1) : kShared + 3 * (cc - 1 - r) + 2);
        sx[cc][t] = ok ? A.X[(size_t)c * A.ldx + k] : 0.f;
    }
    for (int a = 0; a < np; ++a) sv[a][t] = ok ? A.V[(size_t)k * np + a] : 0.f;
    __syncthreads();
    if (ok) {
        float acc = 0.f;
        for (int a = 0; a < np; ++a) acc = fmaf(sv[a][t], szp[a], acc);
        A.vz[k] = acc;
    }
    float* out = A.part + (size_t)blockIdx.x * np * nc;
    for (int pi = t; pi < np * nc; pi += kLinRows) {
        const int a = pi / nc, cc = pi % nc;
        float acc = 0.f;
#pragma unroll 8
        for (int kk = 0; kk < kLinRows; ++kk) acc = fmaf(sv[a][kk], sx[cc][kk], acc);
        out[pi] = acc;
    }
}

__global__ void __launch_bounds__(kLinRows) k_linear(LinArgs A) { linear_impl(A); }

__global__ void __launch_bounds__(kLinRows) k_linear_b(const LinArgs* __restrict__ args) {
    const LinArgs& a = args[blockIdx.z];
    if (a.np <= 0 || (int)blockIdx.x * kLinRows >= a.K) return;
    linear_impl(a);
}

void launch_linear(cudaStream_t s, const LinArgs& a, int n_blocks) {
    k_linear<<<n_blocks, kLinRows, 0, s>>>(a);
}

void launch_linear_batched(cudaStream_t s, const LinArgs* d_args, int n_sys, int max_blocks) {
    if (n_sys > 0 && max_blocks > 0) k_linear_b<<<dim3(max_blocks, 1, n_sys), kLinRows, 0, s>>>(d_args);
}

}  // namespace dae
