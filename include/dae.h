/*
 * dae.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * "High-order Differentiable Autoencoder for Nonlinear Model Reduction"
 * (Shen et al., arXiv 2102.11026).
 *
 * What the library computes, per call, for a fully connected decoder
 * u = D(q) (Sec. 3.5, Fig. 3; hidden activation tanh, sin or none, linear output
 * layer) and a tetrahedral mesh with lumped diagonal mass M (Sec. 3.1, Eq. 1):
 *
 *   Delta = q - qbar,  z = Delta - dt*qbar_dot,  w = 3*Delta - dt*qbar_dot
 *   u = D(q),  J = dD/dq (Eq. 4),  H[qdot,qdot] with qdot = Delta/dt (Eq. 5),
 *   dJ = S[.,Delta,Delta] + H[., w]                                   (Eq. 12)
 *   phi = J^T M (J z + H[Delta,Delta]) + dt^2 J^T (f_C - f_ext)        (Eqs. 7-8)
 *   A   = a^T H + J^T M (J + dJ) + dt^2 sum_{e in C} w_e J_e^T K_e J_e  (Eq. 11, n_p = 0)
 *   a   = M (J z + H[Delta,Delta]) + dt^2 (f_C - f_ext)
 *   f_C = sum_{e in C} w_e f_e(u)   (cubature force, Sec. 5)
 *
 * and the reduced implicit-Euler Newton step A delta = -phi with a backtracking
 * line search.  The right contractions (J, H[Delta,.], dJ, H[Delta,Delta]) come
 * from one stacked complex-step forward pass (Sec. 4.3, Eqs. 16-17); a^T H comes
 * from complex-step backpropagation (Sec. 4.4).  Eq. 11 is evaluated with a "+"
 * sign on the dt^2 H^T (f_int - f_ext) term (the derivative of Eq. 10; the paper
 * prints "-").
 *
 * Conventions
 *   - Layouts: decoder weights W_l are row-major (n_out x n_in); displacement-like
 *     vectors have N = 3V entries, vertex-major (x0,y0,z0,x1,...); N x r matrices
 *     (J, dJ, ...) are column-major (column j = derivative along e_j, contiguous);
 *     r x r matrices are column-major.  q-like vectors are FP64, decoder outputs FP32.
 *   - Residency: every array argument may be host or device memory; the library
 *     detects which with cudaPointerGetAttributes.  Host inputs are copied to the
 *     device, host outputs are copied back and the call then synchronizes the
 *     context's stream.  With device-only arguments a call only enqueues work on
 *     the context's stream (except where noted) and returns.
 *   - Ownership: the caller owns every buffer it passes; the library owns
 *     contexts, decoders and meshes until the matching dae_destroy / dae_free_*.
 *   - Errors: functions return a dae_status and never abort; the message of the
 *     most recent failure on a context is available from dae_last_error.  Errors
 *     raised on the device (non-finite values, inverted tets, bounded waits that
 *     gave up) are recorded in a device status word and reported by the next
 *     call that synchronizes (dae_sync, or any call with host outputs).
 *   - Threads: contexts are independent; one context must not be used from two
 *     host threads at once.
 */
#ifndef DAE_H
#define DAE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dae_ctx dae_ctx;
typedef struct dae_decoder dae_decoder;
typedef struct dae_mesh dae_mesh;

typedef enum {
    DAE_OK = 0,
    DAE_ERR_INVALID_ARG = -1,
    DAE_ERR_CUDA = -2,
    DAE_ERR_OOM = -3,
    DAE_ERR_NOT_CONVERGED = -4,
    DAE_ERR_NONFINITE = -5,
    DAE_ERR_SINGULAR = -6,
    DAE_ERR_INVERTED = -7,
    DAE_ERR_TIMEOUT = -8,
    DAE_ERR_UNSUPPORTED = -9
} dae_status;

/* Hidden-layer activation.  The paper uses sin (Sec. 3.5); tanh is the default
 * of the synthetic workloads; LINEAR makes D affine (H = S = 0). */
typedef enum { DAE_ACT_TANH = 0, DAE_ACT_SIN = 1, DAE_ACT_LINEAR = 2 } dae_act;

/* Arithmetic of the decoder GEMMs (accumulation is always FP32):
 *   FP32    CUDA-core FFMA tiles
 *   TF32    tcgen05 kind::tf32 tensor cores (operands rounded to the nearest TF32)
 *   BF16    tcgen05 kind::f16 with BF16 operands
 *   BF16X3  three BF16 products (hi*hi + hi*lo + lo*hi) per split operand pair */
typedef enum { DAE_FP32 = 0, DAE_TF32 = 1, DAE_BF16 = 2, DAE_BF16X3 = 3 } dae_prec;

/* Constitutive law of the tets (Sec. 5 names StVK; Neo-Hookean is the second
 * law the synthetic workloads use). */
typedef enum { DAE_STVK = 0, DAE_NEOHOOKEAN = 1 } dae_material;

/* Newton options (dae_default_newton_opts fills the defaults shown). */
typedef struct {
    int max_iter;        /* Newton updates per frame (5) */
    int max_evals;       /* evaluation budget per frame incl. backtracking (max_iter + 3) */
    int max_halvings;    /* step halvings per line search (8) */
    double tol;          /* stop when |phi| <= tol * max(1, |phi_0|)  (1e-8) */
    double c_armijo;     /* |phi(alpha)|^2 <= (1 - 2 c alpha) |phi|^2  (1e-4) */
    double h_cs;         /* complex-step size; a power of two keeps the scaling exact (2^-20) */
    double max_step;     /* first trial step of an update capped at |alpha delta|_inf <= max_step
                            (0.5, in latent units; 0 = no cap) */
    double xtol;         /* also stop when the next Newton step is negligible:
                            |delta|_inf <= xtol * max(1, |q|_inf)  (1e-6; 0 = off), delta the
                            Newton step at q or, when q was just accepted, its simplified-Newton
                            estimate -A_prev^{-1} phi(q) from the factors of the previous
                            iterate's Newton matrix (then A is not formed at q) */
} dae_newton_opts;

/* Per-frame outcome of dae_newton_step / dae_rollout. */
typedef struct {
    int iters;           /* accepted Newton updates */
    int evals;           /* evaluations of phi (the derivative pass, cubature, phi); those
                            of trials that start no new Newton step (rejected, converged or
                            stopped) skip the reverse pass and the Newton matrix */
    int converged;       /* 1 if |phi| reached tol or the next step fell below xtol */
    int status;          /* dae_status of the frame (device-side errors included) */
    double phi_norm0;    /* |phi| at the first iterate */
    double phi_norm;     /* |phi| at the returned iterate */
    double energy;       /* cubature elastic energy sum w_e V_e Psi_e at the returned iterate */
    double alpha;        /* last accepted step length */
    int full_evals;      /* evaluations that also formed the Newton matrix A and solved
                            A delta = -phi (complex-step reverse pass included) */
} dae_newton_report;

/* ---------------------------------------------------------------- context -- */

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the per-thread default stream). */
dae_status dae_create(dae_ctx** ctx, int device, void* cuda_stream);
dae_status dae_destroy(dae_ctx* ctx);
/* Message of the most recent failure on ctx ("" if none); valid until the next call. */
const char* dae_last_error(const dae_ctx* ctx);
const char* dae_status_string(dae_status s);
/* Wait for the context's stream; returns (and clears) the device status word. */
dae_status dae_sync(dae_ctx* ctx);
void dae_default_newton_opts(dae_newton_opts* opts);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int dae_version(void);

/* ---------------------------------------------------------------- decoder -- */

/*
 * Upload a decoder with n_layers fully connected layers (Sec. 3.5, Fig. 3):
 * z_l = W_l a_{l-1} + b_l, a_l = act(z_l) for l < n_layers, u = z_{n_layers}.
 *   widths   n_layers+1 ints: widths[0] = r (latent size, 1..32), widths[n_layers] = N
 *            (a multiple of 3 when used with a mesh)
 *   W[l]     row-major widths[l+1] x widths[l] FP32 (host or device)
 *   b[l]     widths[l+1] FP32
 *   prec     arithmetic of the decoder GEMMs (the library keeps FP32 weights and
 *            builds the BF16 hi/lo splits it needs)
 * The library copies the weights; the caller may free its arrays on return.
 * This call synchronizes.  Errors: INVALID_ARG (shapes), OOM, CUDA, UNSUPPORTED
 * (r > 32).
 */
dae_status dae_load_decoder(dae_ctx* ctx, int n_layers, const int* widths,
                            const float* const* W, const float* const* b,
                            dae_act act, dae_prec prec, dae_decoder** out);
dae_status dae_free_decoder(dae_decoder* dec);
/* Change the GEMM arithmetic of a loaded decoder (builds splits if needed; synchronizes). */
dae_status dae_decoder_set_precision(dae_decoder* dec, dae_prec prec);

/* Work decomposition of the persistent layer chains (tensor-core precisions): the
 * hidden layers of the stacked forward pass (dir 0) and of the complex-step reverse pass
 * (dir 1) each run in one persistent launch, a layer cut into 128-row tiles with P CTAs
 * per tile (P = 1, 2, 4 or 8; tiles x P at most the SM count), either as a split of the
 * layer's K loop over the P CTAs (split = P, rep = 1; at least two 64-element k-blocks
 * per CTA) or as P replicated K loops (split = 1, rep = P); each CTA finishes 128/P
 * rows.  A small layer (at most 8 tiles and 64 tile k-blocks) may also run solo
 * (split = 1, rep = 0): all its tiles on CTA 0 while the other CTAs skip it; a run of
 * consecutive solo layers hands its activations from layer to layer inside CTA 0.  A
 * plan is per precision: a precision
 * change returns to the built-in plan.
 * These are scheduling choices only; the paper has no counterpart (its passes are
 * cuBLAS GEMMs, Sec. 6). */

/* The current plan of direction dir: split[l], rep[l] for hidden layers l = 0..n_layers-2
 * (network order in both directions).  Errors: INVALID_ARG, UNSUPPORTED (FP32). */
dae_status dae_decoder_get_chain_plan(const dae_decoder* dec, int dir, int* split, int* rep);
/* Set the plan of direction dir (NULL arrays: the built-in plan).  Every (split, rep)
 * must be one of the candidates above for its layer, else INVALID_ARG.  Synchronizes. */
dae_status dae_decoder_set_chain_plan(dae_decoder* dec, int dir, const int* split, const int* rep);
/* Tile autotuner: for each direction, starting from the current plan, one pass over the
 * layers tries every candidate of a layer and keeps it when the chain's launch time
 * (CUDA events, mean of reps launches) drops by more than 1 %; the final plan is timed
 * against the starting one, interleaved, and kept only if not slower.  ms (optional,
 * 4 doubles): forward chain ms before / after, reverse chain ms before / after.
 * Synchronizes; call it outside stream capture, once per decoder and precision. */
dae_status dae_decoder_autotune(dae_decoder* dec, int reps, double* ms);

/* ------------------------------------------------------------------- mesh -- */

/*
 * Upload a tet mesh (Sec. 3.1: FEM discretisation, lumped mass).
 *   X      3*n_vert FP64 rest positions, vertex-major
 *   tets   4*n_tet vertex indices (int32), positively oriented
 *   vmass  n_vert lumped vertex masses (each repeated on the vertex's 3 DOFs)
 *   E, nu  Young's modulus and Poisson ratio (Lame: mu = E/(2(1+nu)),
 *          lam = E nu / ((1+nu)(1-2nu)))
 * Precomputes Dm^{-1} and rest volumes.  Synchronizes.  Errors: INVALID_ARG
 * (index out of range, degenerate rest tet, nu outside (-1, 0.5)), OOM, CUDA.
 */
dae_status dae_load_mesh(dae_ctx* ctx, int n_vert, const double* X, int n_tet,
                         const int* tets, const double* vmass, dae_material material,
                         double E, double nu, dae_mesh** out);
dae_status dae_free_mesh(dae_mesh* mesh);

/* ------------------------------------------------------ hot-path entries -- */

/*
 * Decoder derivatives at q (Sec. 4.3: one stacked complex-step forward pass).
 *   q, qbar, qbar_dot  r FP64 each; dt > 0 (Sec. 3.2 implicit Euler)
 *   u     N       D(q)
 *   J     N x r   dD/dq                                   (Eq. 4)
 *   Hqq   N       H[qdot, qdot], qdot = (q - qbar)/dt     (Eq. 5's inertial term)
 *   dJ    N x r   S[.,Delta,Delta] + H[., w]              (Eq. 12)
 *   Hw    N x r   H[., w]       (costs one extra pass when requested)
 *   Sdd   N x r   S[.,Delta,Delta] (costs one extra pass when requested)
 * Any output may be NULL (not computed where that saves work).  Errors:
 * INVALID_ARG, CUDA, OOM.
 */
dae_status dae_eval_derivs(dae_ctx* ctx, const dae_decoder* dec, const double* q,
                           const double* qbar, const double* qbar_dot, double dt,
                           float* u, float* J, float* Hqq, float* dJ, float* Hw, float* Sdd);

/*
 * Multicomplex activation of dae_eval_derivs (an ablation of the truncated form).
 * exact = 0 (default): the activation of every stacked number is its multicomplex Taylor
 * expansion with the terms of relative order h_cs^2 dropped (Sec. 4.4, Fig. 5), which
 * lets all perturbations share the real, i2 and i2i3 columns (3r + 4 columns).
 * exact = 1: every perturbation e_j is its own tricomplex number
 * q + h e_j i1 + h Delta (i2 + i3) + h^2 w i2i3 with its own real part (6r + 4 columns),
 * and the activation is evaluated in exact multicomplex arithmetic (Sec. 4.1, Eq. 16;
 * App. A: recursive addition theorems, tanh(X + iY) = (sinh 2X + i sin 2Y)/(cosh 2X +
 * cos 2Y)), in FP32 on the CUDA cores.  The two agree to O(h_cs^2) ~ 1e-12 relative,
 * far below FP32 rounding.  Only the FP32 form, r <= 17 and no linear basis; a
 * precision change sets it back to 0.  Errors: INVALID_ARG, UNSUPPORTED.
 */
dae_status dae_decoder_set_cs_mode(dae_decoder* dec, int exact);

/*
 * Reduced system at q: phi (Eqs. 7-8 times dt^2), A (Eq. 11 with n_p = 0) and
 * the cubature elastic energy sum_e w_e V_e Psi_e(F_e).
 *   cub_tets  n_cub tet indices (distinct), cub_w n_cub non-negative weights (Sec. 5)
 *   f_ext     N FP32 external force, or NULL for zero
 *   phi       r FP64;  A  r x r FP64 column-major;  energy 1 FP64 (any may be NULL)
 *   terms     optional r x r x 4 + r FP64: [a^T H | J^T M J | J^T M dJ | K_r | J^T f_C]
 *             (column-major blocks), or NULL
 * Errors: INVALID_ARG, INVERTED (det F <= 0 at a Neo-Hookean cubature tet),
 * NONFINITE, CUDA.
 */
dae_status dae_assemble_reduced(dae_ctx* ctx, const dae_decoder* dec, const dae_mesh* mesh,
                                int n_cub, const int* cub_tets, const float* cub_w,
                                const double* q, const double* qbar, const double* qbar_dot,
                                double dt, const float* f_ext, double* phi, double* A,
                                double* energy, double* terms);

/*
 * One implicit-Euler frame: Newton iterations on phi(q) = 0 starting from the
 * value in q (commonly qbar + dt*qbar_dot), each solving A delta = -phi in FP64
 * (LU with partial pivoting) with Armijo backtracking on |phi|^2.  All control
 * runs on the device; the host reads only the report.
 *   q     in: first iterate; out: solution (r FP64)
 *   opts  NULL = defaults;  rep  may be NULL (then the call does not synchronize
 *         when every array is on the device; read the report later with
 *         dae_last_report)
 * Errors: INVALID_ARG, INVERTED, NONFINITE, SINGULAR, CUDA.  Not reaching tol
 * within max_iter is reported in rep->converged, not as an error.
 */
dae_status dae_newton_step(dae_ctx* ctx, const dae_decoder* dec, const dae_mesh* mesh,
                           int n_cub, const int* cub_tets, const float* cub_w, double* q,
                           const double* qbar, const double* qbar_dot, double dt,
                           const float* f_ext, const dae_newton_opts* opts,
                           dae_newton_report* rep);

/* Report of the most recent dae_newton_step on ctx (synchronizes). */
dae_status dae_last_report(dae_ctx* ctx, dae_newton_report* rep);

/*
 * Implicit-Euler rollout of n_frames frames (Sec. 3.2): frame f solves phi = 0
 * from q = qbar + dt*qbar_dot with cubature weights cub_w[f*n_cub ...], then sets
 * qbar_dot = (q - qbar)/dt and qbar = q.
 *   q, qdot   in: state before frame 0; out: state after the last frame (r FP64 each)
 *   cub_w     n_frames x n_cub weights (per-frame redraws)
 *   q_traj    optional n_frames x r FP64 trajectory;  reports optional n_frames
 * The frames run back to back on the device with no host round trip.
 */
dae_status dae_rollout(dae_ctx* ctx, const dae_decoder* dec, const dae_mesh* mesh,
                       int n_cub, const int* cub_tets, const float* cub_w, int n_frames,
                       double* q, double* qdot, double dt, const float* f_ext,
                       const dae_newton_opts* opts, double* q_traj,
                       dae_newton_report* reports);

/* ------------------------------------------------------- linear subspace -- */

/*
 * Add a linear (PCA) subspace to a decoder (Sec. 3.3-3.4, Eqs. 9-11):
 * u = U p + (I - U U^T) D(q), the unknown becomes r = [p; q] (np + r entries,
 * np + r <= 32), Jt = [U, (I - U U^T) J], Ht = diag(0, (I - U U^T) H).
 *   U  np x N basis, row a = basis vector a (unit, mutually orthogonal; host or
 *      device; copied).  The filtering layer (I - U U^T) is folded into the output
 *      layer's weights and bias here, once.
 * Afterwards dae_newton_step / dae_rollout / dae_assemble_reduced take and return
 * (np + r)-vectors q = [p; q], qbar, qbar_dot (phi, A, terms are (np + r)-sized) and
 * need the Gram form (a tensor-core precision and 2K <= N), also in a grouped step;
 * dae_eval_derivs still returns the filtered decoder's derivatives (r columns).  Not
 * with a weight network.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
dae_status dae_decoder_attach_linear(dae_decoder* dec, int np, const float* U);

/* ------------------------------------------------------- weight network -- */

/*
 * Attach a cubature weight network W (Sec. 5, "Weight Prediction") to a decoder:
 * the latent is decoded to u = D(q), then four FC layers of widths[0..4]
 * (widths[0] = N, the decoder output; widths[1..3] <= 1024; widths[4] = the mesh's
 * element count), sin after the first three and a square after the last (weights
 * >= 0).  W[l]: row-major widths[l+1] x widths[l], b[l]: widths[l+1] (host or device;
 * copied).  The first layer is composed with the decoder's linear output layer here,
 * A1 (W_L x + b_L) + b1 = (A1 W_L) x + (A1 b_L + b1), so a prediction never forms u.
 * Once attached, dae_newton_step / dae_rollout / dae_assemble_reduced accept
 * cub_w == NULL: the weights of the cubature tets are then predicted at the first
 * iterate of every frame (at q for dae_assemble_reduced) and held for the frame.
 * Replaces a previously attached network.  Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
dae_status dae_decoder_attach_wnet(dae_decoder* dec, const int* widths, const float* const* W,
                                   const float* const* b);

/* Predicted weights w[i] of the elements tet_ids[i], i < n, at latent q (r FP64);
 * arrays host or device; synchronizes when w is a host array. */
dae_status dae_predict_weights(dae_ctx* ctx, const dae_decoder* dec, const double* q, int n,
                               const int* tet_ids, float* w);

/* ------------------------------------------------------ grouped systems -- */

/*
 * One independent reduced system of a grouped Newton step: its own decoder, mesh,
 * cubature set, state and external force (a domain of a substructured model with
 * no coupling between domains; the puffer ball's 320 strings, each with its own
 * depth-8 decoder, in the paper's Sec. 6 "Extensions and More Results").  Arrays as
 * in dae_newton_step (host or device memory):
 *   q          in: first iterate; out: solution (r FP64)
 *   qbar, qbar_dot  r FP64;  cub_tets, cub_w  n_cub each;  f_ext  N FP32 or NULL
 */
typedef struct dae_system {
    const dae_decoder* dec;
    const dae_mesh* mesh;
    int n_cub;
    const int* cub_tets;
    const float* cub_w;
    double* q;
    const double* qbar;
    const double* qbar_dot;
    const float* f_ext;
} dae_system;

/*
 * One implicit-Euler Newton step (as dae_newton_step) of n_sys independent systems
 * at once: each kernel of a Newton evaluation runs once for all systems that are
 * still iterating (the decoder layers of all systems as the stages of one
 * persistent tensor-core launch), and the evaluation loop repeats on the device
 * until every system is done.  Each system keeps its own Newton control (tol,
 * line search, max_evals from opts, shared by all systems).
 *   Requirements: every decoder on ctx, in one tensor-core precision (TF32, BF16
 *   or BF16X3), appearing in at most one system (workspaces are per decoder).  A
 *   system whose decoder has a linear subspace passes (np + r)-vectors q, qbar, qbar_dot
 *   (as in dae_newton_step); one whose decoder has a weight network may pass
 *   cub_w == NULL (weights predicted at its first evaluation).
 *   reports  n_sys reports or NULL (then the call does not synchronize when every
 *            array is on the device).
 * The launch plan and graph are cached while the systems' decoders, meshes, cubature
 * counts, f_ext presence, dt and opts stay the same.
 * Errors: INVALID_ARG, UNSUPPORTED (FP32 decoder), CUDA; with reports, the first
 * failing system's INVERTED / NONFINITE / SINGULAR status.
 */
dae_status dae_newton_step_batched(dae_ctx* ctx, int n_sys, const dae_system* systems,
                                   double dt, const dae_newton_opts* opts,
                                   dae_newton_report* reports);

/*
 * One implicit-Euler Newton step of domains coupled at interfaces (deformation
 * substructuring, Sec. 6, Fig. 1: the paper's cactus and puffer ball; the paper defers
 * the coupling to Barbic & Zhao 2011).  The ties are read as penalty springs of
 * stiffness k_c:
 *   E_c = k_c/2 (sum_pairs |u_d[i] - u_e[j]|^2 + sum_anchors |u_d[i]|^2)
 * where pair (d, i, e, j) says vertex i of domain d and vertex j of domain e coincide at
 * rest, and anchor (d, i) holds vertex i of domain d at its rest position.  The unknown
 * is all domains' latents; domain d's rows are its own Eq. 10 residual with the tie
 * force -dE_c/du_d among its forces (so a^T H carries it), and the Newton matrix adds
 * the tie Hessian: dt^2 k_c J_d[i]^T J_d[i] on the diagonal blocks and
 * -dt^2 k_c J_d[i]^T J_e[j] off them.  One Newton control (tol, Armijo line search on the
 * global |phi|^2, max_step, xtol from opts) for all domains; the step solves the block
 * system over the forest of domains (pairs must join the domains into a forest: every
 * connected component a tree) by block elimination from the leaves, in FP64.
 *   systems   as in dae_newton_step_batched (tensor-core precision, one precision, each
 *             decoder in one system, no linear subspace); q in/out per system
 *   pairs     n_pairs x 4 ints (d, i, e, j), host array;  anchors  n_anchors x 2 ints (d, i)
 *   rep       one report for the whole step (may be NULL); synchronizes
 * u and J at the tie vertices come from the output layer's FP32 weights and input
 * activations.  Errors: INVALID_ARG (indices, pairs within one domain), UNSUPPORTED (a
 * cycle among the domains, FP32, a linear subspace), SINGULAR, INVERTED, NONFINITE, CUDA.
 */
dae_status dae_newton_step_coupled(dae_ctx* ctx, int n_sys, const dae_system* systems,
                                   int n_pairs, const int* pairs, int n_anchors, const int* anchors,
                                   double k_c, double dt, const dae_newton_opts* opts,
                                   dae_newton_report* rep);

/* ------------------------------------------------------- decoder training -- */

/*
 * Gradients of the decoder's first-order derivatives for fitting a decoder: the
 * paper trains its autoencoder with backpropagation (Sec. 4.4 builds on it; Sec. 5
 * fits the networks).  For a batch of B latents q_s the forward gives
 *     u_s = D(q_s),   J_s = dD/dq (q_s)
 * and the backward, given cotangents gu_s (N) and gJ_s (N x r) of a scalar loss,
 * gives dL/dq_s, dL/dW_l and dL/db_l of L = sum_s gu_s.u_s + sum_{s,j} gJ_s[:,j].J_s e_j.
 * The batch is carried as C = B (1 + r) columns (value and the r tangents of each
 * sample), so every layer is one dense GEMM on the tensor cores in split BF16x3 with
 * FP32 accumulation (forward Z = W X, reverse W^T Z̄, weights Z̄ X^T over the C
 * columns).  The backward recomputes the forward, keeping the pre-activations of
 * every second hidden layer and recomputing the others.
 *
 * Layouts: W[l] row-major widths[l+1] x widths[l] FP32, b[l] widths[l+1] FP32 (the
 * caller's current parameters, read on every call); q B x r FP64 row-major;
 * uJ and g_uJ (1 + r) x B x N FP32: block 0 holds u_s (row s), block 1 + j holds
 * J_s e_j; g_q B x r FP64; g_W[l], g_b[l] like W[l], b[l] (overwritten).  All arrays
 * must be device memory (these entries do not stage host arrays).  Calls enqueue on
 * the context's stream and return.  Errors: INVALID_ARG (shapes, B outside
 * 1..max_batch, host arrays), UNSUPPORTED (r > 32), OOM, CUDA.
 */
typedef struct dae_trainer dae_trainer;
dae_status dae_trainer_create(dae_ctx* ctx, int n_layers, const int* widths, dae_act act,
                              int max_batch, dae_trainer** out);
dae_status dae_trainer_free(dae_trainer* t);
/* GEMM arithmetic of the training pass: DAE_BF16X3 (default; tcgen05 tensor cores,
 * three BF16 products per split operand pair, FP32 accumulation) or DAE_FP32 (FFMA on
 * the CUDA cores from FP32 operands, FP32 accumulation).  Synchronizes; errors:
 * UNSUPPORTED (another precision), OOM. */
dae_status dae_trainer_set_precision(dae_trainer* t, dae_prec prec);
dae_status dae_train_forward(dae_trainer* t, const float* const* W, const float* const* b, int B,
                             const double* q, float* uJ);
dae_status dae_train_backward(dae_trainer* t, const float* const* W, const float* const* b, int B,
                              const double* q, const float* g_uJ, double* g_q,
                              float* const* g_W, float* const* g_b);

/* ------------------------------------------------ allocation-free variant -- */

/*
 * The output-row reductions of dae_assemble_reduced, for callers that cannot
 * allocate device memory: processes that hand all device memory to their own
 * pool at start-up, real-time loops where a cudaMalloc stall is not allowed, or
 * code that runs while an allocator is busy.  This entry point calls no
 * cudaMalloc / cudaFree and no allocating library routine: its per-block partial
 * sums live in a fixed file-scope device array of 4 MiB (2^20 floats) plus 32 KiB
 * of FP64 sums, reserved on every GPU that loads this library until the process
 * exits.  The paper has no counterpart; it is an interface for such callers.
 *
 *   N, r         output rows and latent size (1 <= r <= 32)
 *   J, dJ        N x r column-major (as written by dae_eval_derivs)
 *   HDD          N: H[Delta,Delta] (= dt^2 times the Hqq output of dae_eval_derivs)
 *   mdof         N lumped mass per DOF;  f_ext  N external force or NULL
 *   z            r FP32: (q - qbar) - dt qbar_dot
 *   phi_dense    r FP64: J^T (M (J z + H[Delta,Delta]) - dt^2 f_ext)
 *   Mr, B        r x r FP64 column-major: J^T M J and J^T M dJ (either may be NULL)
 *   cuda_stream  stream to enqueue on (NULL = legacy default stream)
 * Every pointer is device memory; the call only enqueues and returns.  Limits:
 * ceil(N / 128) * (r + r(r+1)/2 + r^2) <= 2^20 (for r = 30: N <= 96 000);
 * larger problems return DAE_ERR_INVALID_ARG.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the one array
 * and each call overwrites it, so calls that can overlap on the GPU (different
 * streams, or concurrent host threads) race: serialize them.
 */
dae_status dae_reduce_rows_noalloc(int N, int r, const float* J, const float* dJ,
                                   const float* HDD, const float* mdof, const float* f_ext,
                                   const float* z, double dt, double* phi_dense, double* Mr,
                                   double* B, void* cuda_stream);

/* ------------------------------------------------------ instrumentation -- */
/* Not part of the paper's method: device timing of the phases of every
 * evaluation, for benchmarks and profiles. */
typedef enum {
    DAE_PHASE_FWD_HIDDEN = 0,  /* hidden-layer GEMMs + multicomplex activation */
    DAE_PHASE_FWD_OUT = 1,     /* output-layer GEMM + output epilogue */
    DAE_PHASE_ROWS = 2,        /* J^T M J, J^T M dJ, J^T a row reductions */
    DAE_PHASE_CUBATURE = 3,    /* cubature forces and stiffness */
    DAE_PHASE_WTA = 4,         /* W_L^T a */
    DAE_PHASE_BWD = 5,         /* complex-step reverse pass through the hidden layers */
    DAE_PHASE_ASSEMBLE = 6,    /* FP64 reductions, assembly, LU and Newton control */
    DAE_PHASE_SEED = 7,        /* input columns of the stacked complex-step batch */
    DAE_N_PHASES = 8
} dae_phase;

/* Record a CUDA event pair around every enqueued phase p with bit (1 << p) set in
 * mask (0 = off; (1 << DAE_N_PHASES) - 1 = all phases). */
dae_status dae_profile_enable(dae_ctx* ctx, unsigned mask);
/* Synchronize, then return per phase the summed device time (ms) and the number of
 * recorded phase instances since the previous read (arrays of DAE_N_PHASES). */
dae_status dae_profile_read(dae_ctx* ctx, double* ms, long long* count);
/* Self-test of the device-side bounded waits: launches a kernel whose mbarrier wait
 * and grid-barrier spin can never complete (nothing arrives) and checks that both
 * give up after their limit (2 s each) instead of hanging.  Synchronizes; the
 * context stays usable.  Returns DAE_OK when both waits gave up, DAE_ERR_TIMEOUT if
 * one did not report it. */
dae_status dae_selftest_bounded_waits(dae_ctx* ctx);
/* Number of kernels enqueued on ctx since it was created. */
long long dae_launch_count(const dae_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DAE_H */
