// Coupled domains of a substructured body (deformation substructuring, Sec. 6): the
// domains' own evaluations run as the grouped launches of dae_newton_step_batched; the
// kernels here add the ties and take one Newton step over all domains' latents.
//
// Reading of the paper (it defers the coupling to Barbic & Zhao 2011): penalty ties of
// stiffness k_c between interface vertices that coincide at rest, and anchors holding a
// vertex at rest,
//   E_c = k_c/2 (sum_pairs |u_d[i] - u_e[j]|^2 + sum_anchors |u_d[i]|^2).
// Its gradient g = dE_c/du joins each domain's forces (Eq. 10: phi_d += dt^2 J_d^T g_d;
// the reverse pass's seed a_d += dt^2 g_d, so a^T H carries it), and its Hessian adds
//   A_dd += dt^2 k_c sum_{ties at i} J_d[i]^T J_d[i],   A_de = -dt^2 k_c sum_pairs J_d[i]^T J_e[j]
// (J_d[i]: the 3 rows of J_d at vertex i).  The Newton step solves the block system over
// the forest of domains (pairs join a child to its parent) by block elimination from the
// leaves to the root, one CTA per connected component, in FP64.
#include <math.h>
#include "dae_internal.h"
#include "epilogue.cuh"

namespace dae {

constexpr int kUJ = 1 + kMaxR;   // u and J columns per tie DOF

// u and J at the 3 DOFs of every tie vertex from the output layer's input activations:
// u_n = b_n + W_n . x_0, J_nj = W_n . x_{i1 of j} / h (the real and i1 columns of the
// stacked complex-step batch), FP32 dot products over the K hidden units.
__global__ void __launch_bounds__(128) k_tie_uj(const CoupledArgs* __restrict__ pa) {
    const CoupledArgs& A = *pa;
    const int t = blockIdx.x;
    if (t >= A.n_tv || A.cs->done) return;
    const TieDom& D = A.dom[A.tv_dom[t]];
    const int v = A.tv_vert[t], r = D.r;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float ih = (float)(1.0 / A.h);
    for (int o = warp; o < 3 * (1 + r); o += 4) {
        const int c = o / (1 + r), col = o % (1 + r);
        const int n = 3 * v + c;
        const float* __restrict__ w = D.W + (size_t)n * D.ld;
        const float* __restrict__ x = D.X + (size_t)(col == 0 ? 0 : kShared + 3 * (col - 1)) * D.ldx;
        float s = 0.f;
        for (int k = lane; k < D.K; k += 32) s = fmaf(w[k], x[k], s);
        for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (lane == 0) A.uJ[((size_t)t * 3 + c) * kUJ + col] = col == 0 ? s + D.b[n] : s * ih;
    }
}

void launch_tie_uj(cudaStream_t s, const CoupledArgs* d_args, int n_tv) {
    if (n_tv > 0) k_tie_uj<<<n_tv, 128, 0, s>>>(d_args);
}

// Global Newton state from the domains' first iterates (their states were just set).
__global__ void k_coupled_begin(const CoupledArgs* __restrict__ pa) {
    const CoupledArgs& A = *pa;
    for (int k = threadIdx.x; k < A.n_tot; k += blockDim.x) {
        const TieDom& D = A.dom[A.unk_dom[k]];
        const double q = D.ns->q_trial[k - D.off];
        A.q_acc[k] = q;
        A.q_trial[k] = q;
        A.delta[k] = 0.0;
        A.phi[k] = 0.0;
    }
    if (threadIdx.x == 0) {
        CoupledState& S = *A.cs;
        S.merit_acc = 0.0; S.phi_norm0 = 0.0; S.alpha = 1.0; S.energy = 0.0; S.coupling_energy = 0.0;
        S.halvings = 0; S.iters = 0; S.evals = 0; S.done = 0; S.converged = 0; S.status = 0;
        S.nfull = 0; S.skip = 0;
    }
}

void launch_coupled_begin(cudaStream_t s, const CoupledArgs* d_args) {
    k_coupled_begin<<<1, 256, 0, s>>>(d_args);
}

// Block sum of a double over 256 threads (result on every thread).
__device__ __forceinline__ double block_sum256(double v, double* sh) {
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];   // fixed order: reproducible
    return s;
}

// The domains' states follow the global iterate and decision.
__device__ __forceinline__ void push_states(const CoupledArgs& A) {
    const CoupledState& S = *A.cs;
    for (int k = threadIdx.x; k < A.n_tot; k += blockDim.x) {
        const TieDom& D = A.dom[A.unk_dom[k]];
        D.ns->q_trial[k - D.off] = A.q_trial[k];
        D.ns->q_acc[k - D.off] = A.q_acc[k];
    }
    for (int d = threadIdx.x; d < A.n_dom; d += blockDim.x) {
        NewtonState* ns = A.dom[d].ns;
        ns->done = S.done;
        ns->skip_rev = S.skip;
        ns->evals = S.evals;
        ns->iters = S.iters;
        ns->converged = S.converged;
        ns->status = S.status;
        ns->alpha = S.alpha;
    }
}

// Tie forces, the global phi and the line-search decision on the global |phi|^2
// (Armijo with halving, as for one domain).  Runs after every domain's phi and energy
// (k_decide in assemble-only mode) and before the reverse pass, whose seed gets the tie
// forces as extra (DOF, force) pairs.
__global__ void __launch_bounds__(256) k_coupled_decide(const CoupledArgs* __restrict__ pa) {
    const CoupledArgs& A = *pa;
    CoupledState& S = *A.cs;
    if (S.done) return;
    __shared__ double sh[8];
    __shared__ int s_bad, s_nonfinite;
    __shared__ int s_dec;
    const int t0 = threadIdx.x;
    if (t0 == 0) { s_bad = 0; s_nonfinite = 0; }
    __syncthreads();
    // g at the tie vertices and the coupling energy
    double ec = 0.0;
    for (int t = t0; t < A.n_tv; t += blockDim.x) {
        const float* ut = A.uJ + (size_t)t * 3 * kUJ;
        const double na = A.n_anch[t];
        const TieDom& D = A.dom[A.tv_dom[t]];
        const int v = A.tv_vert[t], slot = A.tv_slot[t];
        for (int c = 0; c < 3; ++c) {
            const double u = ut[c * kUJ];
            double g = na * u, e = na * u * u;
            for (int m = A.nb_off[t]; m < A.nb_off[t + 1]; ++m) {
                const double du = u - (double)A.uJ[((size_t)A.nb[m] * 3 + c) * kUJ];
                g += du;
                e += 0.5 * du * du;   // each pair is seen from both of its vertices
            }
            g *= A.kc;
            A.g[(size_t)t * 3 + c] = g;
            ec += 0.5 * A.kc * e;
            D.fe_w[D.pair0 + 3 * slot + c] = (float)g;
            D.fe_dof[D.pair0 + 3 * slot + c] = 3 * v + c;
        }
    }
    ec = block_sum256(ec, sh);
    // the domains' flags (inverted tet / bad cubature index) and energies
    for (int d = t0; d < A.n_dom; d += blockDim.x) {
        const TieDom& D = A.dom[d];
        const int f = *D.eval_flag;
        if (f) atomicMax(&s_bad, f == 2 ? 2 : 1);
        *D.eval_flag = 0;
    }
    double en = 0.0;
    for (int d = t0; d < A.n_dom; d += blockDim.x) {
        const TieDom& D = A.dom[d];
        en += D.red[D.r + D.r * D.r];
    }
    en = block_sum256(en, sh);
    // phi_d + dt^2 J_d^T g_d
    const double dt2 = A.dt * A.dt;
    double m2 = 0.0;
    for (int k = t0; k < A.n_tot; k += blockDim.x) {
        const int d = A.unk_dom[k];
        const TieDom& D = A.dom[d];
        const int i = k - D.off;
        double p = D.red[i];
        for (int m = A.dtv_off[d]; m < A.dtv_off[d + 1]; ++m) {
            const int t = A.dtv[m];
            for (int c = 0; c < 3; ++c)
                p += dt2 * (double)A.uJ[((size_t)t * 3 + c) * kUJ + 1 + i] * A.g[(size_t)t * 3 + c];
        }
        if (!isfinite(p)) s_nonfinite = 1;
        A.phi[k] = p;       // of the trial; becomes the accepted phi when accepted
        m2 += p * p;
    }
    const double merit = block_sum256(m2, sh);
    if (t0 == 0) {
        S.evals += 1;
        const int flag = s_bad;
        const bool bad = flag || s_nonfinite || !isfinite(merit);
        int dec;   // 0 reject, 1 accept-and-continue, 2 accept-and-stop, 3 stop
        if (S.evals == 1) {
            if (bad) {
                S.status = flag == 2 ? DAE_ERR_INVALID_ARG : (flag ? DAE_ERR_INVERTED : DAE_ERR_NONFINITE);
                dec = 3;
            } else {
                S.phi_norm0 = sqrt(merit);
                dec = 1;
            }
        } else {
            const bool ok = !bad && merit <= (1.0 - 2.0 * A.c_armijo * S.alpha) * S.merit_acc;
            dec = ok ? 1 : 0;
        }
        if (dec == 1) {
            S.merit_acc = merit;
            S.energy = en + ec;
            S.coupling_energy = ec;
            if (S.evals > 1) S.iters += 1;
            if (sqrt(merit) <= A.tol * fmax(1.0, S.phi_norm0)) { S.converged = 1; dec = 2; }
            else if (S.iters >= A.max_iter) dec = 2;
        } else if (dec == 0) {
            if (S.halvings >= A.max_halvings) dec = 3;
        }
        if ((dec == 0 || dec == 1) && S.evals >= A.max_evals) dec = 3;
        if (dec == 1) {
            S.skip = 0;
            S.nfull += 1;
        } else if (dec == 0) {
            S.skip = 1;
            S.alpha *= 0.5;
            S.halvings += 1;
        } else {
            S.skip = 1;
            S.done = 1;
        }
        s_dec = dec;
    }
    __syncthreads();
    const int dec = s_dec;
    for (int k = t0; k < A.n_tot; k += blockDim.x) {
        if (dec == 1 || dec == 2) A.q_acc[k] = A.q_trial[k];
        else if (dec == 0) A.q_trial[k] = A.q_acc[k] + S.alpha * A.delta[k];
    }
    __syncthreads();
    push_states(A);
}

void launch_coupled_decide(cudaStream_t s, const CoupledArgs* d_args) {
    k_coupled_decide<<<1, 256, 0, s>>>(d_args);
}

// --------------------------------------------------------- block solve --
// In-place LU with partial pivoting of the r x r matrix S (shared, row stride 33) by
// 256 threads; piv[k] = row swapped with row k.  Returns false when a pivot is below
// 1e-13 max|S| (the coupled Newton matrix is then reported singular).
__device__ bool lu_factor(double (*S)[33], int* piv, int r) {
    __shared__ double s_max;
    __shared__ int s_p, s_ok;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (warp == 0) {
        double m = 0.0;
        for (int i = lane; i < r * r; i += 32) m = fmax(m, fabs(S[i / r][i % r]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) { s_max = m; s_ok = m > 0.0 && isfinite(m); }
    }
    __syncthreads();
    for (int k = 0; k < r && s_ok; ++k) {
        if (warp == 0) {
            double v = (lane >= k && lane < r) ? fabs(S[lane][k]) : -1.0;
            int idx = lane;
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
                if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
            }
            if (lane == 0) {
                s_p = idx;
                piv[k] = idx;
                if (!(v > 1e-13 * s_max)) s_ok = 0;
            }
        }
        __syncthreads();
        if (!s_ok) break;
        const int p = s_p;
        if (p != k && t < r) { const double a = S[k][t]; S[k][t] = S[p][t]; S[p][t] = a; }
        __syncthreads();
        const double inv = 1.0 / S[k][k];
        if (t > k && t < r) S[t][k] *= inv;
        __syncthreads();
        const int m = r - k - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            S[i][j] = fma(-S[i][k], S[k][j], S[i][j]);
        }
        __syncthreads();
    }
    __syncthreads();
    return s_ok != 0;
}

// B (r x m, shared, row stride 33) <- S^{-1} B with the factors of lu_factor; one
// thread per right-hand side.
__device__ void lu_solve(const double (*S)[33], const int* piv, int r, double (*B)[33], int m) {
    const int c = threadIdx.x;
    if (c < m) {
        for (int k = 0; k < r; ++k) {
            const int p = piv[k];
            if (p != k) { const double a = B[k][c]; B[k][c] = B[p][c]; B[p][c] = a; }
        }
        for (int i = 1; i < r; ++i) {
            double s = B[i][c];
            for (int k = 0; k < i; ++k) s = fma(-S[i][k], B[k][c], s);
            B[i][c] = s;
        }
        for (int i = r - 1; i >= 0; --i) {
            double s = B[i][c];
            for (int k = i + 1; k < r; ++k) s = fma(-S[i][k], B[k][c], s);
            B[i][c] = s / S[i][i];
        }
    }
    __syncthreads();
}

// One CTA per connected component of the domain forest: the global Newton step
// A delta = -phi by block elimination, children before parents:
//   S_c = A_cc (+ Schur updates from c's children), y_c = S_c^{-1} b_c,
//   X_c = S_c^{-1} A_cp,  S_p -= A_cp^T X_c,  b_p -= A_cp^T y_c        (A_pc = A_cp^T)
// then delta_root = y_root and, parents before children, delta_c = y_c - X_c delta_p.
__global__ void __launch_bounds__(256) k_coupled_solve(const CoupledArgs* __restrict__ pa) {
    const CoupledArgs& A = *pa;
    const CoupledState& St = *A.cs;
    if (St.done || St.skip) return;
    __shared__ double S[kMaxR][33], B[kMaxR][33], C[kMaxR][33];
    __shared__ int piv[kMaxR];
    const int comp = blockIdx.x, t = threadIdx.x;
    const int o0 = A.comp_off[comp], o1 = A.comp_off[comp + 1];
    const double ck = A.dt * A.dt * A.kc;
    // S_d = A_dd + dt^2 k_c sum_{tie vertices of d} deg J^T J,  y_d = -phi_d
    for (int o = o0; o < o1; ++o) {
        const int d = A.order[o];
        const TieDom& D = A.dom[d];
        const int r = D.r;
        double* Sd = A.S + (size_t)d * kMaxR * kMaxR;
        for (int e = t; e < r * r; e += blockDim.x) {
            const int i = e / r, j = e % r;
            double s = D.red[r + j * r + i];
            for (int m = A.dtv_off[d]; m < A.dtv_off[d + 1]; ++m) {
                const int tv = A.dtv[m];
                const double deg = A.n_anch[tv] + (A.nb_off[tv + 1] - A.nb_off[tv]);
                const float* u = A.uJ + (size_t)tv * 3 * kUJ;
                double jj = 0.0;
                for (int c = 0; c < 3; ++c) jj += (double)u[c * kUJ + 1 + i] * (double)u[c * kUJ + 1 + j];
                s += ck * deg * jj;
            }
            Sd[i * kMaxR + j] = s;
        }
        for (int i = t; i < r; i += blockDim.x) A.y[(size_t)d * kMaxR + i] = -A.phi[D.off + i];
    }
    __syncthreads();
    int ok = 1;
    for (int o = o0; o < o1 && ok; ++o) {
        const int d = A.order[o];
        const int r = A.dom[d].r, p = A.parent[d];
        double* Sd = A.S + (size_t)d * kMaxR * kMaxR;
        for (int e = t; e < r * r; e += blockDim.x) S[e / r][e % r] = Sd[(e / r) * kMaxR + e % r];
        for (int i = t; i < r; i += blockDim.x) B[i][0] = A.y[(size_t)d * kMaxR + i];
        __syncthreads();
        if (!lu_factor(S, piv, r)) { ok = 0; break; }
        // the child's coupling block A_cp (r x rp) into C, then X = S^{-1} [A_cp | b]
        const int rp = p >= 0 ? A.dom[p].r : 0;
        if (p >= 0) {
            for (int e = t; e < r * rp; e += blockDim.x) {
                const int i = e / rp, j = e % rp;
                double s = 0.0;
                for (int m = A.cp_off[d]; m < A.cp_off[d + 1]; ++m) {
                    const float* ua = A.uJ + (size_t)A.cp[2 * m] * 3 * kUJ;
                    const float* ub = A.uJ + (size_t)A.cp[2 * m + 1] * 3 * kUJ;
                    for (int c = 0; c < 3; ++c) s += (double)ua[c * kUJ + 1 + i] * (double)ub[c * kUJ + 1 + j];
                }
                C[i][j] = -ck * s;
                B[i][1 + j] = C[i][j];
            }
        }
        __syncthreads();
        lu_solve(S, piv, r, B, 1 + rp);
        for (int i = t; i < r; i += blockDim.x) A.y[(size_t)d * kMaxR + i] = B[i][0];
        if (p >= 0) {
            double* Xd = A.X + (size_t)d * kMaxR * kMaxR;
            for (int e = t; e < r * rp; e += blockDim.x) Xd[(e / rp) * kMaxR + e % rp] = B[e / rp][1 + e % rp];
            // S_p -= C^T X,  y_p -= C^T y
            double* Sp = A.S + (size_t)p * kMaxR * kMaxR;
            for (int e = t; e < rp * rp; e += blockDim.x) {
                const int i = e / rp, j = e % rp;
                double s = 0.0;
                for (int k = 0; k < r; ++k) s = fma(C[k][i], B[k][1 + j], s);
                Sp[i * kMaxR + j] -= s;
            }
            for (int i = t; i < rp; i += blockDim.x) {
                double s = 0.0;
                for (int k = 0; k < r; ++k) s = fma(C[k][i], B[k][0], s);
                A.y[(size_t)p * kMaxR + i] -= s;
            }
        }
        __syncthreads();
    }
    if (!ok) {
        if (t == 0) atomicCAS(&A.cs->status, 0, (int)DAE_ERR_SINGULAR);
        return;
    }
    // back substitution, root first
    for (int o = o1 - 1; o >= o0; --o) {
        const int d = A.order[o];
        const TieDom& D = A.dom[d];
        const int r = D.r, p = A.parent[d];
        const int rp = p >= 0 ? A.dom[p].r : 0;
        const double* Xd = A.X + (size_t)d * kMaxR * kMaxR;
        for (int i = t; i < r; i += blockDim.x) {
            double s = A.y[(size_t)d * kMaxR + i];
            if (p >= 0)
                for (int j = 0; j < rp; ++j) s = fma(-Xd[i * kMaxR + j], A.delta[A.dom[p].off + j], s);
            A.delta[D.off + i] = s;
        }
        __syncthreads();
    }
}

void launch_coupled_solve(cudaStream_t s, const CoupledArgs* d_args, int n_comp) {
    if (n_comp > 0) k_coupled_solve<<<n_comp, 256, 0, s>>>(d_args);
}

// After the solve: the step test |delta|_inf <= xtol max(1, |q|_inf), the first-trial
// cap |alpha delta|_inf <= max_step, the next trial, and the domains' states.
__global__ void __launch_bounds__(256) k_coupled_update(const CoupledArgs* __restrict__ pa) {
    const CoupledArgs& A = *pa;
    CoupledState& S = *A.cs;
    if (S.done || S.skip) return;
    __shared__ double sh[8];
    __shared__ double s_xn, s_qn;
    double xn = 0.0, qn = 0.0;
    for (int k = threadIdx.x; k < A.n_tot; k += blockDim.x) {
        xn = fmax(xn, fabs(A.delta[k]));
        qn = fmax(qn, fabs(A.q_acc[k]));
    }
    for (int m = 16; m > 0; m >>= 1) {
        xn = fmax(xn, __shfl_xor_sync(0xffffffffu, xn, m));
        qn = fmax(qn, __shfl_xor_sync(0xffffffffu, qn, m));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = xn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w) a = fmax(a, sh[w]);
        s_xn = a;
    }
    __syncthreads();
    if (lane == 0) sh[warp] = qn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w) a = fmax(a, sh[w]);
        s_qn = a;
        if (S.status) {
            S.done = 1;
        } else if (A.xtol > 0.0 && s_xn <= A.xtol * fmax(1.0, s_qn)) {
            S.converged = 1;
            S.done = 1;
        } else {
            S.alpha = (A.max_step > 0.0 && s_xn > A.max_step) ? A.max_step / s_xn : 1.0;
            S.halvings = 0;
        }
    }
    __syncthreads();
    if (!S.done)
        for (int k = threadIdx.x; k < A.n_tot; k += blockDim.x) A.q_trial[k] = A.q_acc[k] + S.alpha * A.delta[k];
    __syncthreads();
    push_states(A);
}

void launch_coupled_update(cudaStream_t s, const CoupledArgs* d_args) {
    k_coupled_update<<<1, 256, 0, s>>>(d_args);
}

}  // namespace dae
