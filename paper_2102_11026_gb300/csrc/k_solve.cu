// FP64 assembly of the reduced system (Eqs. 10-11 with n_p = 0), the dense
// LU solve of the Newton step and the device-side Newton / line-search control.
#include <math.h>
#include <string.h>
#include "dae_internal.h"
#include "epilogue.cuh"

namespace dae {

// out[e] = sum_p part[p * stride + e] for e < n_ent, in FP64; 32 threads per entry
// with a fixed summation tree (bitwise reproducible).
// out[e] = sum_p part[p][e].  A block takes 32 consecutive entries (the lanes,
// coalesced loads); warp w of 16 sums the parts p = w (mod 16): each group of four
// of its terms is summed in FP32 and added to an FP64 accumulator (FP64 adds are
// scarce on this part), then the 16 warp sums are added in warp order (fixed order:
// bitwise reproducible).
__device__ __forceinline__ void colsum_impl(const float* part, int n_parts, int stride,
                                            int n_ent, double* out, const NewtonState* ns) {
    if (ns && ns->done) return;
    __shared__ double ws[16][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (e < n_ent) {
        int p = w;
        for (; p + 48 < n_parts; p += 64) {
            const float a = part[(size_t)p * stride + e];
            const float b = part[(size_t)(p + 16) * stride + e];
            const float c = part[(size_t)(p + 32) * stride + e];
            const float d = part[(size_t)(p + 48) * stride + e];
            acc += (double)((a + b) + (c + d));
        }
        for (; p < n_parts; p += 16) acc += (double)part[(size_t)p * stride + e];
    }
    ws[w][lane] = acc;
    __syncthreads();
    if (w == 0 && e < n_ent) {
        double s = 0.0;
        for (int q = 0; q < 16; ++q) s += ws[q][lane];
        out[e] = s;
    }
}

__global__ void __launch_bounds__(512) k_colsum(const float* part, int n_parts, int stride,
                                                int n_ent, double* out, const NewtonState* ns) {
    colsum_impl(part, n_parts, stride, n_ent, out, ns);
}

__device__ __forceinline__ void dsum_impl(const double* x, int n, double* out,
                                          const NewtonState* ns) {
    if (ns && ns->done) return;
    __shared__ double s[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_dsum(const double* x, int n, double* out, const NewtonState* ns) {
    dsum_impl(x, n, out, ns);
}


__device__ __forceinline__ int upper_idx(int i, int j, int r) {
    if (i > j) { int t = i; i = j; j = t; }
    return i * r - i * (i - 1) / 2 + (j - i);
}

// Solve A x = b in FP64 accuracy (r <= 32, A column-major FP64, in shared memory) by
// mixed-precision iterative refinement (Wilkinson; Moler 1967): LU with partial
// pivoting of the FP32-rounded A, then x <- x + U^{-1} L^{-1} P (b - A x) with the
// residual formed in FP64.  Each correction shrinks the error by about
// kappa(A) r eps_32, so kRefine corrections reach FP64 rounding for the reduced
// Newton matrices (kappa ~ 1e1 - 1e3).  FP64 issue is scarce on this part (each
// dependent FP64 operation costs ~100 cycles; an FP64 LU took ~60 us of latency),
// so the factorisation runs in FP32.
//   LU: the FP32-rounded A in shared memory, row i in row i; per column k warp 0 picks
//   the pivot row among the rows not yet used (largest |.|, lowest index on ties)
//   without swapping rows, the 128 threads update the other unused rows' columns
//   right of k, and the multipliers replace column k.  Warp 0 then holds row i of the
//   factors in lane i's registers for the triangular solves.
// Called by the 128 threads of warps 0-3.  Returns 0, or DAE_ERR_SINGULAR when an
// FP32 pivot is below 2^-20 max|A| (such A are beyond what the FP32 factors resolve).
constexpr int kRefine = 3;
constexpr int kCtlThreads = 256;   // threads of k_control (its assembly assumes this count)

// One warp: d = U^{-1} L^{-1} P b in FP32 with the factors of mixed_solve (lane i holds
// row i of the factors, the step ps at which it was the pivot, and b_i); returns d_i on
// lane i.  Branch-free chains: steps past r are no-ops (perm 0, multiplier 0).
__device__ __forceinline__ float lu_apply(const float* row, int ps, const int* pk, const float* rk,
                                          float bv, int r) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kMaxR; ++k) {
        const float bp = __shfl_sync(full, bv, pk[k]);
        const float m = (k < r && ps > k) ? row[k] : 0.f;
        bv = fmaf(-m, bp, bv);
    }
    float d = 0.f;
#pragma unroll
    for (int k = kMaxR - 1; k >= 0; --k) {
        const float xk = __shfl_sync(full, bv, pk[k]) * rk[k];
        if (lane == k) d = xk;
        const float m = (k < r && ps >= 0 && ps < k) ? row[k] : 0.f;
        bv = fmaf(-m, xk, bv);
    }
    return d;
}

// Layout of the stored FP32 factors (lu_out of mixed_solve): [32][32] rows, then ps,
// perm and 1/pivot per row (floats; perm and ps exact small integers).
constexpr int kLuRows = 0, kLuPs = kMaxR * kMaxR, kLuPerm = kLuPs + kMaxR, kLuRinv = kLuPerm + kMaxR;
constexpr int kLuFloats = kLuRinv + kMaxR;

__device__ int mixed_solve(const double* A, const double* b, double* x, int r, float* lu_out) {
    __shared__ int perm[kMaxR];
    __shared__ float rinv[kMaxR], dsol[kMaxR];
    __shared__ double res[kMaxR], part[4][kMaxR];
    __shared__ int s_sing, s_p;
    __shared__ unsigned s_used;
    __shared__ int s_ps[kMaxR];
    __shared__ float F[kMaxR][kMaxR + 1];   // the FP32 factors in place, row i = row i of A
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned full = 0xffffffffu;
    float row[kMaxR];   // warp 0: row `lane` of the factors (L left of its pivot step, U from it)
    int ps = -1;        // warp 0: the elimination step at which row `lane` was the pivot
    if (t < r) { x[t] = 0.0; res[t] = b[t]; }
    for (int e = t; e < kMaxR * kMaxR; e += 128) {
        const int i = e & (kMaxR - 1), j = e / kMaxR;
        F[i][j] = (i < r && j < r) ? (float)A[(size_t)j * r + i] : 0.f;
    }
    if (t < kMaxR) s_ps[t] = -1;
    if (t == 0) { s_used = 0u; s_sing = 0; }
    asm volatile("bar.sync 2, 128;" ::: "memory");
    float am = 0.f;
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < kMaxR; ++j) am = fmaxf(am, fabsf(F[lane][j]));
        for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(full, am, o));
    }
    // LU with partial pivoting, no row swaps: per column k warp 0 picks the pivot row among
    // the rows not yet used, then the 128 threads update the other unused rows (thread
    // (lane, warp) takes row lane, columns k+1+warp, k+5+warp, ...), then the multipliers
    // replace column k.  Column k+1 is updated by warp 0, which searches it next.
    for (int k = 0; k < r; ++k) {
        if (warp == 0) {
            const unsigned used = s_used;
            const float v = F[lane][k];
            // the largest |v| among the unused rows in one warp reduction.  Key: the bits
            // of |v| (non-negative floats order like unsigned integers) with the low 5
            // mantissa bits replaced by 31 - lane, so among values equal to 2^-18 relative
            // the lowest row wins (any of them is a sound partial pivot; the FP64
            // refinement below fixes the solution's accuracy)
            const unsigned key = (lane < r && !((used >> lane) & 1u))
                                     ? ((__float_as_uint(fabsf(v)) & ~31u) | (31u - (unsigned)lane))
                                     : 0u;
            const unsigned best = __reduce_max_sync(full, key);
            const int p = 31 - (int)(best & 31u);
            const float pv = __uint_as_float(best & ~31u);
            if (lane == 0) {
                if (!(pv > 0x1p-20f * am) || !isfinite(pv)) {
                    s_sing = 1;
                } else {
                    perm[k] = p;
                    rinv[k] = __frcp_rn(F[p][k]);
                    s_ps[p] = k;
                    s_used = used | (1u << p);
                    s_p = p;
                }
            }
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (s_sing) break;
        const int p = s_p;
        const bool act = lane < r && !((s_used >> lane) & 1u);
        const float l = act ? F[lane][k] * rinv[k] : 0.f;
        if (act) {
            // this thread's (<= 8) columns: every operand load in flight before the stores
            // (row p is not written at step k, row `lane` only by its own threads)
            float fp[kMaxR / 4], fl[kMaxR / 4];
#pragma unroll
            for (int u = 0; u < kMaxR / 4; ++u) {
                const int j = k + 1 + warp + 4 * u;
                if (j < r) { fp[u] = F[p][j]; fl[u] = F[lane][j]; }
            }
#pragma unroll
            for (int u = 0; u < kMaxR / 4; ++u) {
                const int j = k + 1 + warp + 4 * u;
                if (j < r) F[lane][j] = fmaf(-l, fp[u], fl[u]);
            }
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (warp == 0 && act) F[lane][k] = l;
        __syncwarp();
    }
    if (s_sing) return DAE_ERR_SINGULAR;
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < kMaxR; ++j) row[j] = F[lane][j];
        ps = s_ps[lane];
    }
    if (lu_out && warp == 0) {
        // the factors for the next iterate's simplified-Newton step estimate (k_decide)
#pragma unroll
        for (int j = 0; j < kMaxR; ++j) lu_out[kLuRows + lane * kMaxR + j] = row[j];
        lu_out[kLuPs + lane] = (float)ps;
        lu_out[kLuPerm + lane] = lane < r ? (float)perm[lane] : 0.f;
        lu_out[kLuRinv + lane] = lane < r ? rinv[lane] : 0.f;
    }
    for (int it = 0; it <= kRefine; ++it) {
        if (warp == 0) {
            // d = U^{-1} L^{-1} P res in FP32; lane i holds the right-hand side of row i
            int pk[kMaxR];
            float rk[kMaxR];
#pragma unroll
            for (int k = 0; k < kMaxR; ++k) {
                pk[k] = k < r ? perm[k] : 0;
                rk[k] = k < r ? rinv[k] : 0.f;
            }
            const float d = lu_apply(row, ps, pk, rk, lane < r ? (float)res[lane] : 0.f, r);
            if (lane < r) dsol[lane] = d;
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (t < r) x[t] += (double)dsol[t];
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (it == kRefine) break;
        // res = b - A x in FP64: thread (i, c) sums the columns j = c (mod 4) of row i
        {
            const int i = lane, c = warp;
            double sacc = 0.0;
            if (i < r)
                for (int j = c; j < r; j += 4) sacc = fma(A[(size_t)j * r + i], x[j], sacc);
            part[c][i] = sacc;
        }
        asm volatile("bar.sync 2, 128;" ::: "memory");
        if (t < r) res[t] = b[t] - ((part[0][t] + part[1][t]) + (part[2][t] + part[3][t]));
        asm volatile("bar.sync 2, 128;" ::: "memory");
    }
    return 0;
}

// The FP64 end of one evaluation, in two kernels around the reverse pass.
//   rowsum  [phi_dense (rq) | Mr upper | B (i*rq+j)]
//   cubsum  [g_int (r) | K_r upper]
//   bwd     [(1+rq) x rq] per split: column 0 = J^T a, column 1+j = h (a^T H)[:, j]
//   red     [phi (r) | A (r*r col-major) | energy | aH | Mr | B | Kr | g_int]
// k_decide forms phi (Eqs. 7-8 times dt^2, Eq. 10 with a linear subspace) and the
// energy, and under Newton control takes the line-search decision on the iterate just
// evaluated (Armijo on |phi|^2, reading R6): accept it (a new Newton step follows,
// unless it converged), or reject it and halve the step.  Only an accepted,
// unconverged iterate needs the Newton matrix, so every other evaluation sets
// ns->skip_rev and its reverse pass, W_L^T a and the solve are skipped: those are
// phi-only evaluations.  k_control then forms A (Eq. 11) and solves A delta = -phi.

// Linear subspace (np > 0): unknowns [p; q], decoder partials over rq = r - np.
struct LinView {
    const CtlArgs& C;
    int rq, nc;
    double inv_h, inv_h3;
    __device__ double umj(int a, int j) const { return C.linsum[a * nc + 1 + j] * inv_h; }          // U^T M J
    __device__ double umdj(int a, int j) const { return C.linsum[a * nc + 1 + rq + j] * inv_h3; }   // U^T M dJ
};

__device__ __forceinline__ void decide_impl(const CtlArgs& C) {
    if (C.ns && C.ns->done) return;
    __shared__ double sphi[kMaxR];
    __shared__ double szp[kMaxR], szq[kMaxR];
    __shared__ int nonfinite;
    __shared__ double s_merit;
    __shared__ __align__(8) NewtonState S;
    const int r = C.r, t = threadIdx.x;
    const double dt2 = C.dt * C.dt;
    const double inv_h = 1.0 / C.h;   // one divide (exact for power-of-two steps)
    double* phi = C.red;
    double* energy = C.red + r + r * r;
    double* gint = energy + 1 + 4 * r * r;
    if (t == 0) nonfinite = 0;
    if (C.control) {
        const int nw = sizeof(NewtonState) / sizeof(int);
        for (int i = t; i < nw; i += blockDim.x)
            reinterpret_cast<int*>(&S)[i] = reinterpret_cast<const int*>(C.ns)[i];
    }
    __syncthreads();
    const int np = C.np, rq = np > 0 ? C.rq : r;
    const LinView lv{C, rq, 1 + 2 * rq, inv_h, inv_h * inv_h * inv_h};
    if (np > 0) {
        const double* qe = C.control ? S.q_trial : C.q_in;
        for (int i = t; i < r; i += blockDim.x) {
            const double z = (qe[i] - C.qbar[i]) - C.dt * C.qbar_dot[i];
            if (i < np) szp[i] = z; else szq[i - np] = z;
        }
        __syncthreads();
    }
    for (int i = t; i < r; i += blockDim.x) {
        const double g = C.have_cub ? C.cubsum[i] : 0.0;
        gint[i] = g;
        double p;
        if (i >= np) {
            // J^T (M y_q - dt^2 f_ext) + J^T M U z_p + dt^2 J^T f_C
            const int qi = i - np;
            p = C.rowsum[qi] + dt2 * g;
            for (int a = 0; a < np; ++a) p += lv.umj(a, qi) * szp[a];
        } else {
            // U^T M U z_p + U^T M (H[D,D] + J z_q) + dt^2 U^T (f_C - f_ext)
            p = C.linsum[i * lv.nc] * inv_h * inv_h + dt2 * (g - (C.Uf ? (double)C.Uf[i] : 0.0));
            for (int b = 0; b < np; ++b) p += (double)C.UMU[i * np + b] * szp[b];
            for (int j = 0; j < rq; ++j) p += lv.umj(i, j) * szq[j];
        }
        phi[i] = p;
        sphi[i] = p;
        if (!isfinite(p)) nonfinite = 1;
    }
    const double en = C.have_cub ? *C.esum : 0.0;
    if (t == 0) *energy = en;
    __syncthreads();
    if (!C.control) return;   // statuses of an assemble-only call: k_control
    // |phi|^2 by a warp reduction (serial FP64 chains are slow on this part), and the
    // simplified-Newton estimate of the step from this iterate, -A_prev^{-1} phi, with the
    // FP32 factors of the last Newton matrix (reading R6: a frame whose estimated next
    // step is below xtol stops here, without forming A at this iterate)
    __shared__ double s_est, s_qn;
    __shared__ int s_est_ok;
    if (t < 32) {
        double m2 = t < r ? sphi[t] * sphi[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        if (t == 0) s_merit = m2;
        const bool est = C.lu && S.lu_ok && C.xtol > 0.0;
        if (est) {
            float row[kMaxR], rk[kMaxR];
            int pk[kMaxR];
#pragma unroll
            for (int j = 0; j < kMaxR; ++j) {
                row[j] = C.lu[kLuRows + t * kMaxR + j];
                pk[j] = (int)C.lu[kLuPerm + j];
                rk[j] = C.lu[kLuRinv + j];
            }
            const int ps = (int)C.lu[kLuPs + t];
            const float d = lu_apply(row, ps, pk, rk, t < r ? (float)(-sphi[t]) : 0.f, r);
            double xn = (t < r && isfinite(d)) ? fabs((double)d) : (t < r ? INFINITY : 0.0);
            double qn = t < r ? fabs(S.q_trial[t]) : 0.0;
            for (int o = 16; o > 0; o >>= 1) {
                xn = fmax(xn, __shfl_xor_sync(0xffffffffu, xn, o));
                qn = fmax(qn, __shfl_xor_sync(0xffffffffu, qn, o));
            }
            if (t == 0) { s_est = xn; s_qn = qn; }
        }
        if (t == 0) s_est_ok = est ? 1 : 0;
    }
    __syncthreads();
    if (t == 0) {
        const int flag = C.eval_flag ? *C.eval_flag : 0;   // 1 inverted tet, 2 bad cubature index
        const bool inverted = flag != 0;
        S.evals += 1;
        const double merit = s_merit;
        const bool bad = inverted || nonfinite || !isfinite(merit);
        int dec;   // 0 reject, 1 accept-and-continue, 2 accept-and-stop, 3 stop
        if (S.evals == 1) {
            if (bad) {
                S.status = flag == 2 ? DAE_ERR_INVALID_ARG
                         : (inverted ? DAE_ERR_INVERTED : DAE_ERR_NONFINITE);
                dec = 3;
            } else {
                S.phi_norm0 = sqrt(merit);
                dec = 1;
            }
        } else {
            const bool ok = !bad && merit <= (1.0 - 2.0 * C.c_armijo * S.alpha) * S.merit_acc;
            dec = ok ? 1 : 0;
        }
        if (dec == 1) {
            for (int i = 0; i < r; ++i) { S.q_acc[i] = S.q_trial[i]; S.phi[i] = sphi[i]; }
            S.merit_acc = merit;
            S.energy = en;
            if (S.evals > 1) S.iters += 1;
            const double pn = sqrt(merit);
            if (pn <= C.tol * fmax(1.0, S.phi_norm0)) { S.converged = 1; dec = 2; }
            else if (S.iters >= C.max_iter) dec = 2;
            else if (S.evals > 1 && s_est_ok && s_est <= C.xtol * fmax(1.0, s_qn)) { S.converged = 1; dec = 2; }
        } else if (dec == 0) {
            if (S.halvings >= C.max_halvings) dec = 3;
        }
        if ((dec == 0 || dec == 1) && S.evals >= C.max_evals) dec = 3;
        if (dec == 1) {
            S.skip_rev = 0;
            S.nfull += 1;
        } else if (dec == 0) {
            S.skip_rev = 1;
            S.alpha *= 0.5;
            S.halvings += 1;
            for (int i = 0; i < r; ++i) S.q_trial[i] = S.q_acc[i] + S.alpha * S.delta[i];
        } else {
            S.skip_rev = 1;
            S.done = 1;
        }
        if (C.eval_flag) *C.eval_flag = 0;
        if (C.kcount) atomicAdd(C.kcount, (unsigned long long)C.kpe);
    }
    __syncthreads();
    const int nw = sizeof(NewtonState) / sizeof(int);
    for (int i = t; i < nw; i += blockDim.x)
        reinterpret_cast<int*>(C.ns)[i] = reinterpret_cast<const int*>(&S)[i];
}

__global__ void k_decide(CtlArgs C) { decide_impl(C); }

__device__ __forceinline__ void control_impl(const CtlArgs& C) {
    const int t = threadIdx.x;
    if (C.ns && (C.ns->done || C.ns->skip_rev)) {
        // no Newton step from this evaluation: the loop ends once the frame is done
        if (C.use_cond && t == 0) cudaGraphSetConditional(C.hcond, C.ns->done ? 0u : 1u);
        return;
    }
    __shared__ double rhs[kMaxR];
    __shared__ double x[kMaxR];
    __shared__ int nonfinite;
    __shared__ double sbwd[(kMaxR + 1) * kMaxR];
    __shared__ double sA[kMaxR * kMaxR];   // A for the solve's residuals
    __shared__ __align__(8) NewtonState S;
    const int r = C.r;
    const double dt2 = C.dt * C.dt;
    const double inv_h = 1.0 / C.h;
    double* phi = C.red;
    double* A = C.red + r;
    double* energy = C.red + r + r * r;
    double* aH = energy + 1;
    double* Mr = aH + r * r;
    double* Bm = Mr + r * r;
    double* Kr = Bm + r * r;
    if (t == 0) nonfinite = 0;
    if (C.control) {
        const int nw = sizeof(NewtonState) / sizeof(int);
        for (int i = t; i < nw; i += blockDim.x)
            reinterpret_cast<int*>(&S)[i] = reinterpret_cast<const int*>(C.ns)[i];
    }
    const int np = C.np, rq = np > 0 ? C.rq : r, nsq = rq * (rq + 1) / 2;
    const LinView lv{C, rq, 1 + 2 * rq, inv_h, inv_h * inv_h * inv_h};
    // column sums of the reverse pass's partials (one per split), in FP64
    const int nb = (1 + rq) * rq;
    for (int e = t; e < nb; e += blockDim.x) {
        double acc = 0.0;
        for (int p = 0; p < C.bwd_split; ++p) acc += (double)C.bwd_part[(size_t)p * nb + e];
        sbwd[e] = acc;
    }
    __syncthreads();
    // thread t assembles the elements e = t + kCtlThreads u: every term of its elements
    // is loaded before the first store (the column sums and the terms are disjoint
    // regions of one buffer, which the compiler cannot tell)
    constexpr int kAsmIt = (kMaxR * kMaxR + kCtlThreads - 1) / kCtlThreads;
    double v_ah[kAsmIt], v_mr[kAsmIt], v_b[kAsmIt], v_kr[kAsmIt];
#pragma unroll
    for (int u = 0; u < kAsmIt; ++u) {
        const int e = t + kCtlThreads * u;
        double ah = 0.0, mr = 0.0, b = 0.0, kr = 0.0;
        if (e < r * r) {
            const int i = e % r, j = e / r;   // column-major (i, j)
            if (i >= np && j >= np) {
                const int qi = i - np, qj = j - np;
                ah = 0.5 * inv_h * (sbwd[(1 + qj) * rq + qi] + sbwd[(1 + qi) * rq + qj]);
                mr = C.rowsum[rq + upper_idx(qi, qj, rq)];
                b = C.rowsum[rq + nsq + qi * rq + qj];
            } else if (i < np && j < np) {
                mr = (double)C.UMU[i * np + j];              // U^T M U
            } else if (i < np) {
                mr = lv.umj(i, j - np);                      // U^T M [J + dJ]
                b = lv.umdj(i, j - np);
            } else {
                mr = lv.umj(j, i - np);                      // J^T M U
            }
            if (C.have_cub) kr = C.cubsum[r + upper_idx(i, j, r)];
        }
        v_ah[u] = ah; v_mr[u] = mr; v_b[u] = b; v_kr[u] = kr;
    }
#pragma unroll
    for (int u = 0; u < kAsmIt; ++u) {
        const int e = t + kCtlThreads * u;
        if (e < r * r) {
            const double a = v_ah[u] + v_mr[u] + v_b[u] + dt2 * v_kr[u];
            aH[e] = v_ah[u]; Mr[e] = v_mr[u]; Bm[e] = v_b[u]; Kr[e] = v_kr[u];
            A[e] = a;
            sA[e] = a;
            if (!isfinite(a)) nonfinite = 1;
        }
    }
    if (!C.control) {
        for (int i = t; i < r; i += blockDim.x)
            if (!isfinite(phi[i])) nonfinite = 1;
        __syncthreads();
        if (t == 0) {
            const int flag = C.eval_flag ? *C.eval_flag : 0;
            if (flag == 2) set_status(C.status, DAE_ERR_INVALID_ARG);
            else if (flag) set_status(C.status, DAE_ERR_INVERTED);
            else if (nonfinite) set_status(C.status, DAE_ERR_NONFINITE);
            if (C.eval_flag) *C.eval_flag = 0;
        }
        return;
    }
    for (int i = t; i < r; i += blockDim.x) rhs[i] = -S.phi[i];
    __syncthreads();
    __shared__ double s_xn, s_qn;
    __shared__ int lu_st;
    if (nonfinite) {
        if (t == 0) lu_st = DAE_ERR_NONFINITE;
    } else if (t < 128) {
        const int st0 = mixed_solve(sA, rhs, x, r, C.lu);
        if (t == 0) lu_st = st0;
    }
    __syncthreads();
    const int st = lu_st;
    if (t < 32) {
        double xn = (t < r && !st) ? fabs(x[t]) : 0.0, qn = t < r ? fabs(S.q_acc[t]) : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            xn = fmax(xn, __shfl_xor_sync(0xffffffffu, xn, o));
            qn = fmax(qn, __shfl_xor_sync(0xffffffffu, qn, o));
        }
        if (t == 0) { s_xn = xn; s_qn = qn; }
    }
    __syncthreads();
    if (t == 0) {
        if (st) {
            S.status = st;
            S.done = 1;
        } else {
            const double xn = s_xn, qn = s_qn;
            if (C.xtol > 0.0 && xn <= C.xtol * fmax(1.0, qn)) {
                // the remaining correction is negligible: q_acc is the solution
                S.converged = 1;
                S.done = 1;
            } else {
                // the first trial step is capped at max_step in the max-norm
                S.alpha = (C.max_step > 0.0 && xn > C.max_step) ? C.max_step / xn : 1.0;
                S.halvings = 0;
                S.lu_ok = C.lu ? 1 : 0;
            }
        }
    }
    __syncthreads();
    if (!st && !S.done)
        for (int i = t; i < r; i += blockDim.x) {
            S.delta[i] = x[i];
            S.q_trial[i] = S.q_acc[i] + S.alpha * x[i];
        }
    __syncthreads();
    if (t == 0 && C.use_cond) cudaGraphSetConditional(C.hcond, S.done ? 0u : 1u);
    const int nw = sizeof(NewtonState) / sizeof(int);
    for (int i = t; i < nw; i += blockDim.x)
        reinterpret_cast<int*>(C.ns)[i] = reinterpret_cast<const int*>(&S)[i];
}

__global__ void k_control(CtlArgs C) { control_impl(C); }

void assemble_parts(const AsmArgs& a, ColsumArgs cs[4], DsumArgs& ds, CtlArgs& c) {
    const int r = a.r;                       // system size (np + rq)
    const int np = a.np, rq = np > 0 ? a.rq : r;
    const int nsym = r * (r + 1) / 2, nsq = rq * (rq + 1) / 2;
    // scratch doubles live after the terms block of red
    double* base = a.red + (r + r * r + 1 + 4 * r * r + r);
    double* rowsum = base;
    double* cubsum = rowsum + (r + nsym + r * r);
    double* bwdsum = cubsum + (r + nsym);
    double* esum = bwdsum + (1 + r) * r;
    double* linsum = esum + 1;
    cs[0] = ColsumArgs{a.row_part, a.n_row_blocks, a.row_stride, rq + nsq + rq * rq, rowsum, a.ns};
    cs[1] = ColsumArgs{a.cub_part, a.cub_parts, a.cub_stride, a.n_cub > 0 ? r + nsym : 0, cubsum, a.ns};
    // the reverse pass's partials are summed by k_control (the reverse pass may be skipped)
    cs[2] = ColsumArgs{nullptr, 0, 0, 0, bwdsum, a.ns};
    cs[3] = ColsumArgs{a.lin_part, a.lin_blocks, np * (1 + 2 * rq), np > 0 ? np * (1 + 2 * rq) : 0,
                       linsum, a.ns};
    ds = DsumArgs{a.cub_energy, a.n_cub > 0 ? a.cub_parts : 0, esum, a.ns};
    memset(&c, 0, sizeof c);
    c.r = r; c.dt = a.dt; c.h = a.h;
    c.rowsum = rowsum; c.cubsum = cubsum; c.esum = esum;
    c.bwd_part = a.bwd_part; c.bwd_split = a.bwd_split;
    c.have_cub = a.n_cub > 0;
    c.red = a.red; c.ns = a.ns; c.control = a.control;
    c.tol = a.tol; c.c_armijo = a.c_armijo; c.max_step = a.max_step; c.xtol = a.xtol; c.max_iter = a.max_iter;
    c.max_halvings = a.max_halvings; c.max_evals = a.max_evals;
    c.eval_flag = a.eval_flag; c.status = a.status; c.lu = a.lu;
    c.hcond = a.hcond; c.use_cond = a.use_cond; c.kcount = a.kcount; c.kpe = a.kpe;
    c.rq = rq; c.np = np; c.linsum = linsum; c.UMU = a.UMU; c.Uf = a.Uf;
    c.qbar = a.qbar; c.qbar_dot = a.qbar_dot; c.q_in = a.q_in;
}

// The column sums of one evaluation in one launch (y = which sum; an empty sum skips);
// block (0, 4) forms the energy sum.
struct ColsumPack { ColsumArgs cs[4]; DsumArgs ds; };
__global__ void __launch_bounds__(512) k_colsum4(const ColsumPack P) {
    if (blockIdx.y == 4) {
        // energy: every thread of the block takes part (tree in shared memory)
        if (blockIdx.x != 0 || P.ds.n <= 0 || (P.ds.ns && P.ds.ns->done)) return;
        __shared__ double sd[512];
        const int t = threadIdx.x;
        double acc = 0.0;
        for (int i = t; i < P.ds.n; i += 512) acc += P.ds.x[i];
        sd[t] = acc;
        __syncthreads();
        for (int o = 256; o > 0; o >>= 1) {
            if (t < o) sd[t] += sd[t + o];
            __syncthreads();
        }
        if (t == 0) *P.ds.out = sd[0];
        return;
    }
    const ColsumArgs& a = P.cs[blockIdx.y];
    if ((int)blockIdx.x * 32 >= a.n_ent) return;
    colsum_impl(a.part, a.n_parts, a.stride, a.n_ent, a.out, a.ns);
}

void launch_decide(cudaStream_t s, const AsmArgs& a) {
    ColsumPack P;
    CtlArgs c;
    assemble_parts(a, P.cs, P.ds, c);
    if (a.n_cub <= 0) { P.cs[1].n_ent = 0; P.ds.n = 0; }
    int max_ent = 1;
    for (int i = 0; i < 4; ++i) max_ent = P.cs[i].n_ent > max_ent ? P.cs[i].n_ent : max_ent;
    k_colsum4<<<dim3((max_ent + 31) / 32, 5), 512, 0, s>>>(P);
    k_decide<<<1, 64, 0, s>>>(c);
}

void launch_control(cudaStream_t s, const AsmArgs& a) {
    ColsumArgs cs[4];
    DsumArgs ds;
    CtlArgs c;
    assemble_parts(a, cs, ds, c);
    k_control<<<1, kCtlThreads, 0, s>>>(c);
}

// Grouped form: z = system; the column sums in y (an empty sum skips), then the energy
// sum and the decision, one block per system; the control step after the reverse pass.
__global__ void __launch_bounds__(512) k_colsum_b(const ColsumArgs* __restrict__ cs) {
    const ColsumArgs& a = cs[blockIdx.z * 4 + blockIdx.y];
    if ((int)blockIdx.x * 32 >= a.n_ent) return;
    colsum_impl(a.part, a.n_parts, a.stride, a.n_ent, a.out, a.ns);
}
__global__ void k_dsum_b(const DsumArgs* __restrict__ ds) {
    const DsumArgs& a = ds[blockIdx.x];
    if (a.n <= 0) return;
    dsum_impl(a.x, a.n, a.out, a.ns);
}
__global__ void k_decide_b(const CtlArgs* __restrict__ c) { decide_impl(c[blockIdx.x]); }
__global__ void k_control_b(const CtlArgs* __restrict__ c) { control_impl(c[blockIdx.x]); }

void launch_decide_batched(cudaStream_t s, const ColsumArgs* cs, const DsumArgs* ds,
                           const CtlArgs* c, int n_sys, int max_ent) {
    if (n_sys <= 0) return;
    k_colsum_b<<<dim3((max_ent + 31) / 32, 4, n_sys), 512, 0, s>>>(cs);
    k_dsum_b<<<n_sys, 256, 0, s>>>(ds);
    k_decide_b<<<n_sys, 64, 0, s>>>(c);
}

void launch_control_batched(cudaStream_t s, const CtlArgs* c, int n_sys) {
    if (n_sys <= 0) return;
    k_control_b<<<n_sys, kCtlThreads, 0, s>>>(c);
}

// --------------------------------------------------------- frame control --
// A frame (Sec. 3.2 implicit Euler): first iterate q0 = qbar + dt qbar_dot (or a
// given q), Newton evaluations until k_control marks it done, then the update
// qbar_dot <- (q - qbar)/dt, qbar <- q.  Inside a graph the two loops are
// conditional WHILE nodes driven by these kernels and k_control.
__global__ void k_roll_setup(RollCtl* rc, int n_frames, int given_q0, int advance,
                             const double* q_in, int r) {
    const int i = threadIdx.x;
    if (i < r) rc->q_in[i] = given_q0 ? q_in[i] : 0.0;
    if (i == 0) {
        rc->n_frames = n_frames;
        rc->frame = 0;
        rc->given_q0 = given_q0;
        rc->advance = advance;
    }
}

__global__ void k_roll_init(RollCtl* rc, cudaGraphConditionalHandle h, int use,
                            unsigned long long* kcount) {
    rc->frame = 0;
    if (kcount) atomicAdd(kcount, 1ull);
    if (use) cudaGraphSetConditional(h, rc->n_frames > 0 ? 1u : 0u);
}

__global__ void k_frame_start(RollCtl* rc, NewtonState* ns, const double* qbar,
                              const double* qbar_dot, double dt, int r,
                              cudaGraphConditionalHandle h, int use, unsigned long long* kcount) {
    const int i = threadIdx.x;
    if (i < r) {
        const double q0 = rc->given_q0 ? rc->q_in[i] : qbar[i] + dt * qbar_dot[i];
        ns->q_trial[i] = q0;
        ns->q_acc[i] = q0;
        ns->delta[i] = 0.0;
        ns->phi[i] = 0.0;
    }
    if (i == 0) {
        ns->merit_acc = 0.0; ns->phi_norm0 = 0.0; ns->alpha = 1.0; ns->energy = 0.0;
        ns->halvings = 0; ns->iters = 0; ns->evals = 0; ns->done = 0; ns->converged = 0;
        ns->skip_rev = 0; ns->nfull = 0; ns->lu_ok = 0;
        ns->status = 0; ns->frame = rc->frame;
        if (kcount) atomicAdd(kcount, 1ull);
        if (use) cudaGraphSetConditional(h, 1u);
    }
}

__global__ void k_frame_finish(RollCtl* rc, NewtonState* ns, double* qbar, double* qbar_dot,
                               double dt, int r, double* traj, NewtonState* hist, double* q_out,
                               cudaGraphConditionalHandle h, int use, unsigned long long* kcount) {
    const int i = threadIdx.x;
    const int f = rc->frame;
    if (i < r) {
        const double q = ns->q_acc[i];
        q_out[i] = q;
        if (rc->advance) {
            qbar_dot[i] = (q - qbar[i]) / dt;
            qbar[i] = q;
        }
        if (traj) traj[(size_t)f * r + i] = q;
    }
    __syncthreads();
    if (i == 0) {
        ns->done = 1;
        if (hist) hist[f] = *ns;
        rc->frame = f + 1;
        if (kcount) atomicAdd(kcount, 1ull);
        if (use) cudaGraphSetConditional(h, (f + 1 < rc->n_frames) ? 1u : 0u);
    }
}

void launch_roll_setup(cudaStream_t s, RollCtl* rc, int n_frames, int given_q0, int advance,
                       const double* q_in, int r) {
    k_roll_setup<<<1, 32, 0, s>>>(rc, n_frames, given_q0, advance, q_in, r);
}
void launch_roll_init(cudaStream_t s, RollCtl* rc, cudaGraphConditionalHandle h, int use,
                      unsigned long long* kcount) {
    k_roll_init<<<1, 1, 0, s>>>(rc, h, use, kcount);
}
void launch_frame_start(cudaStream_t s, RollCtl* rc, NewtonState* ns, const double* qbar,
                        const double* qbar_dot, double dt, int r, cudaGraphConditionalHandle h,
                        int use, unsigned long long* kcount) {
    k_frame_start<<<1, 32, 0, s>>>(rc, ns, qbar, qbar_dot, dt, r, h, use, kcount);
}
void launch_frame_finish(cudaStream_t s, RollCtl* rc, NewtonState* ns, double* qbar,
                         double* qbar_dot, double dt, int r, double* traj, NewtonState* hist,
                         double* q_out, cudaGraphConditionalHandle h, int use,
                         unsigned long long* kcount) {
    k_frame_finish<<<1, 32, 0, s>>>(rc, ns, qbar, qbar_dot, dt, r, traj, hist, q_out, h, use,
                                    kcount);
}

// Grouped single-frame control: one block per system.  Begin: Newton state from the
// given first iterate (and the evaluation loop's condition set); end: the accepted
// iterate out.  The condition kernel keeps the loop going while any system runs.
__global__ void k_frame_begin_b(const FrameArgs* __restrict__ f, cudaGraphConditionalHandle h,
                                int use) {
    const FrameArgs& a = f[blockIdx.x];
    NewtonState* ns = a.ns;
    const int i = threadIdx.x;
    if (i < a.r) {
        const double q0 = a.q0[i];
        ns->q_trial[i] = q0;
        ns->q_acc[i] = q0;
        ns->delta[i] = 0.0;
        ns->phi[i] = 0.0;
    }
    if (i == 0) {
        ns->merit_acc = 0.0; ns->phi_norm0 = 0.0; ns->alpha = 1.0; ns->energy = 0.0;
        ns->halvings = 0; ns->iters = 0; ns->evals = 0; ns->done = 0; ns->converged = 0;
        ns->skip_rev = 0; ns->nfull = 0; ns->lu_ok = 0;
        ns->status = 0; ns->frame = 0;
        if (use && blockIdx.x == 0) cudaGraphSetConditional(h, 1u);
    }
}

__global__ void k_frame_end_b(const FrameArgs* __restrict__ f) {
    const FrameArgs& a = f[blockIdx.x];
    const int i = threadIdx.x;
    if (i < a.r) a.q_out[i] = a.ns->q_acc[i];
    __syncthreads();
    if (i == 0) a.ns->done = 1;
}

__global__ void k_batch_cond(const FrameArgs* __restrict__ f, int n_sys,
                             cudaGraphConditionalHandle h, int use, int* flag) {
    int run = 0;
    for (int i = threadIdx.x; i < n_sys; i += blockDim.x) run |= f[i].ns->done ? 0 : 1;
    run = __syncthreads_or(run);
    if (threadIdx.x == 0) {
        if (use) cudaGraphSetConditional(h, run ? 1u : 0u);
        if (flag) *flag = run;
    }
}

void launch_frame_begin_batched(cudaStream_t s, const FrameArgs* f, int n_sys,
                                cudaGraphConditionalHandle h, int use) {
    k_frame_begin_b<<<n_sys, 32, 0, s>>>(f, h, use);
}
void launch_frame_end_batched(cudaStream_t s, const FrameArgs* f, int n_sys) {
    k_frame_end_b<<<n_sys, 32, 0, s>>>(f);
}
void launch_batch_cond(cudaStream_t s, const FrameArgs* f, int n_sys, cudaGraphConditionalHandle h,
                       int* flag) {
    k_batch_cond<<<1, 256, 0, s>>>(f, n_sys, h, flag ? 0 : 1, flag);
}

// One block per copy; 16-byte vectors where both ends and the size allow it.
__global__ void k_copy_batch(const CopyDesc* __restrict__ d) {
    const CopyDesc c = d[blockIdx.x];
    const uintptr_t a = (uintptr_t)c.src | (uintptr_t)c.dst | (uintptr_t)c.n;
    if ((a & 15) == 0) {
        const uint4* src = reinterpret_cast<const uint4*>(c.src);
        uint4* dst = reinterpret_cast<uint4*>(c.dst);
        for (unsigned long long i = threadIdx.x; i < c.n / 16; i += blockDim.x) dst[i] = src[i];
    } else {
        const unsigned char* src = reinterpret_cast<const unsigned char*>(c.src);
        unsigned char* dst = reinterpret_cast<unsigned char*>(c.dst);
        for (unsigned long long i = threadIdx.x; i < c.n; i += blockDim.x) dst[i] = src[i];
    }
}

void launch_copy_batch(cudaStream_t s, const CopyDesc* d, int n) {
    if (n > 0) k_copy_batch<<<n, 256, 0, s>>>(d);
}

}  // namespace dae
