// Internal declarations of the sm_103a library behind include/dae.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "dae.h"

namespace dae {

// Stacked component columns of one complex-step forward pass (Sec. 4.3).
// The network input is the multicomplex vector
//     q* = q + h e_j i1 + h c i2 + h c i3 + h^2 g i2i3          (one j per group)
// with c = Delta and g = w by default.  Components shared by every j are stored
// once; the i2 and i3 parts are equal (same seed), so are the i1i2 and i1i3 parts:
//   col 0        real part                     -> u
//   col 1        i2 (= i3) part                -> h   J c
//   col 2        i2i3 part                     -> h^2 (J g + H[c,c])
//   col 3        i2i3 part of the group without the g seed -> h^2 H[c,c]
//   col 4+3j     i1 part of group j            -> h   J e_j
//   col 5+3j     i1i2 (= i1i3) part of group j -> h^2 H[e_j, c]
//   col 6+3j     i1i2i3 part of group j        -> h^3 (S[e_j,c,c] + H[e_j,g])  (= dJ e_j, Eq. 12)
constexpr int kShared = 4;
__host__ __device__ inline int n_cols(int r) { return kShared + 3 * r; }
__host__ __device__ inline int pad_cols(int r) { return (n_cols(r) + 15) / 16 * 16; }
// Exact (untruncated) multicomplex columns, an ablation of the shared-column form: column
// 0 the unperturbed input (u = D(q)), columns 1-3 the number q + h Delta (i2 + i3) as
// [real, i2 (= i3), i2i3] (H[D,D]), then per latent direction j six columns at
// kSharedX + 6j: the tricomplex number q + h e_j i1 + h Delta (i2 + i3) + h^2 w i2i3 as
// [real, i1, i2 (= i3), i1i2 (= i1i3), i2i3, i1i2i3]; every group carries its own real
// part (which differs from D(q) by O(h^2)).
constexpr int kSharedX = 4;
__host__ __device__ inline int n_cols_exact(int r) { return kSharedX + 6 * r; }
__host__ __device__ inline int pad_cols_exact(int r) { return (n_cols_exact(r) + 15) / 16 * 16; }
constexpr int kMaxRExact = 17;   // 6r + 4 columns within the FP32 kernel's 112
constexpr int kMaxR = 32;
constexpr int kRowTile = 128;     // output rows per tile (tcgen05 M, SIMT uses 64)
constexpr int kKPad = 64;         // K padding (128 bytes of BF16)
constexpr int kMaxPairSplits = 512;   // cubature-row splits of the W_L^T a GEMV

enum SeedMode { SEED_FULL = 0, SEED_SDD = 1, SEED_HW = 2 };
// activation store mode (after 0 FP32, 1 + BF16 hi, 2 + BF16 hi/lo): FP32 rounded to TF32
constexpr int kStoreTF32 = 3;

struct Layer {
    int n_in = 0, n_out = 0;
    int ld = 0;            // padded row stride of W (elements), multiple of kKPad
    int m_pad = 0;         // n_out padded to kRowTile
    float* W = nullptr;    // [m_pad][ld] FP32, zero padded
    float* b = nullptr;    // [n_out]
    __nv_bfloat16* Wh = nullptr;   // BF16 hi split [m_pad][ld]
    __nv_bfloat16* Wl = nullptr;   // BF16 lo split (W - hi)
    float* Wr = nullptr;           // W rounded to TF32 (operand of the tf32 GEMMs)
    CUtensorMap tm[4];             // TMA maps: A (W or W hi), A lo, B (input activations), B lo
    bool tm_ok = false;
    // transposed copy for the tensor-core reverse pass (hidden layers): [mT_pad][ldT]
    int ldT = 0, mT_pad = 0;
    float* WT = nullptr;
    __nv_bfloat16* WTh = nullptr;
    __nv_bfloat16* WTl = nullptr;
    float* WTr = nullptr;          // W^T rounded to TF32
    CUtensorMap tmR[4];
    bool tmR_ok = false;
};

// Device-resident Newton control state of one frame.
struct NewtonState {
    double q_acc[kMaxR];     // last accepted iterate
    double q_trial[kMaxR];   // iterate being evaluated
    double delta[kMaxR];     // Newton direction from q_acc
    double phi[kMaxR];       // phi at q_trial
    double merit_acc;        // |phi|^2 at q_acc
    double phi_norm0;
    double alpha;
    double energy;
    int halvings;
    int iters;
    int evals;
    int done;                // 1: the remaining evaluations of the frame are skipped
    int converged;
    int status;              // dae_status of the frame
    int frame;
    int skip_rev;            // 1: this evaluation's trial is not accepted for a new Newton
                             //    step (rejected, converged or stopped), so the reverse pass
                             //    and the Newton matrix are skipped (set by k_decide)
    int nfull;               // evaluations of the frame that formed the Newton matrix
    int lu_ok;               // 1: the FP32 factors of the last Newton matrix are stored
};

struct ChainJob;
struct GridBar;

// Device-resident control of a sequence of frames (rollout or single Newton step).
struct RollCtl {
    int n_frames;
    int frame;
    int given_q0;            // 1: first iterate from q_in; 0: qbar + dt qbar_dot
    int advance;             // 1: qbar_dot <- (q - qbar)/dt, qbar <- q after each frame
    double q_in[kMaxR];
};

// Everything a captured frame graph bakes into its kernel parameters.
struct GraphKey {
    unsigned long long mesh_id;
    unsigned long long dec_id;   // bumped by every precision change (the chains are rebuilt)
    const void* cub_w; const void* cub_tets; const void* fe_w; const void* hist; const void* traj;
    const void* fext; const void* gs; const void* wn;
    int n_cub, gram, prec, max_iter, max_halvings, max_evals;
    double dt, h, tol, c_armijo, max_step, xtol;
};

// Per-decoder workspace (sized for the decoder's widths and latent size).
struct Workspace {
    int Cp = 0, C = 0;
    size_t ldx_max = 0;            // max padded width over all layer inputs/outputs
    float* X[2] = {nullptr, nullptr};             // FP32 activations [Cp][ld]
    float* Xe[2] = {nullptr, nullptr};            // exact multicomplex columns [Cpx][ld] (on demand)
    int Cpx = 0;
    __nv_bfloat16* Xh[2] = {nullptr, nullptr};    // BF16 hi [Cp][ld]
    __nv_bfloat16* Xl[2] = {nullptr, nullptr};    // BF16 lo [Cp][ld]
    std::vector<float*> S1;        // per hidden layer: act'(z) [n]
    std::vector<float*> T;         // per hidden layer: act''(z) * (i1 part of z)/h  [r][n]
    // last-layer outputs (internal copies)
    float* u = nullptr;            // [N]
    float* J = nullptr;            // [r][N]
    float* dJ = nullptr;           // [r][N]
    float* HDD = nullptr;          // [N]  H[Delta,Delta]
    float* a = nullptr;            // [N]  dense part of the BP seed: M(Jz+HDD) - dt^2 f_ext
    // per-tile partial sums of the row reductions (FP32)
    float* row_part = nullptr;     // [n_row_blocks][row_stride]
    int n_row_blocks = 0, row_stride = 0;
    // reverse pass partials [nsplit][1+r][width]
    float* bwd_part[2] = {nullptr, nullptr};
    size_t bwd_part_elems = 0;
    float* gbuf = nullptr;         // [1+r][max width] reverse-pass seed of one layer
    // reverse-pass B operands on the tensor-core path: g of one layer, [Cb][ld] (ping-pong)
    int Cb = 0;
    size_t ldg_max = 0;
    float* G32[2] = {nullptr, nullptr};
    __nv_bfloat16* Gh[2] = {nullptr, nullptr};
    __nv_bfloat16* Gl[2] = {nullptr, nullptr};
    // persistent layer-chain jobs (tensor-core precisions)
    ChainJob* fwd_jobs = nullptr;  // hidden forward layers 0..L-2 (device)
    ChainJob* rev_jobs = nullptr;  // reverse layers L-2..0 (device)
    ChainJob* out_job = nullptr;   // output layer, rewritten per call (device)
    GridBar* gbar = nullptr;
    float* chain_part = nullptr;   // split-K partial tiles of the chains
    unsigned* chain_cnt = nullptr;  // per-tile arrival counters of the chains (zero between launches)
    size_t chain_cnt_n = 0;
    unsigned long long sync_epoch = 0;   // ctx->timeout_epoch when gbar / chain_cnt were last valid
    bool chain_ok = false;
    float* split_part = nullptr;   // split-K partial tiles of the hidden tensor-core GEMMs
    int* split_cnt = nullptr;      // per-tile counters
    int max_split = 0;
    // cubature scratch (grown on demand)
    int cub_cap = 0;
    float* fe_w = nullptr;          // [cap][12] w_e f_e
    int* fe_dof = nullptr;          // [cap][12] DOF index
    float* cub_part = nullptr;      // [cap][cub_stride]
    double* cub_energy = nullptr;   // [cap]
    int cub_stride = 0;
    // reduced system (FP64)
    double* red = nullptr;          // phi | A | energy | terms (see dae_assemble_reduced)
    NewtonState* ns = nullptr;
    float* lu = nullptr;            // FP32 factors of the last Newton matrix (step estimate)
    double* qbar = nullptr;         // [r]
    double* qbar_dot = nullptr;     // [r]
    float* zvec = nullptr;          // [r] z = Delta - dt qbar_dot (FP32 copy)
    int* cub_tets = nullptr;        // staged cubature indices
    float* cub_w = nullptr;         // staged weights (per frame)
    int cub_w_cap = 0;
    float* f_ext = nullptr;         // staged f_ext [N] (zero if absent)
    double* q0 = nullptr;           // [r] first iterate of a rollout frame
    int* eval_flag = nullptr;       // per-evaluation cubature flag
    NewtonState* hist = nullptr;    // per-frame states of a rollout (grown on demand)
    int hist_cap = 0;
    double* traj = nullptr;         // [hist_cap][r] accepted iterate of every frame
    double* qout = nullptr;         // [r] result of the last frame
    RollCtl* rc = nullptr;
    // cached frame graph
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    int kpe = 0;                    // kernels per evaluation
    bool graph_ok = false;
    // Gram matrix G = W_L^T M W_L of the output layer for the mesh masses (W_L^T M y = G x_y)
    float* G = nullptr;             // [K][ldG]
    int ldG = 0;
    unsigned long long G_mesh = 0;  // id of the mesh G was formed for
    float* xy = nullptr;            // [K] x_y: y = J z + H[D,D] = W_L x_y
    // W_L^T f_ext, recomputed only when f_ext changes
    float* pext = nullptr;          // [K]
    float* fext_prev = nullptr;     // [N]
    int* pext_flag = nullptr;       // 1: recompute
    bool pext_valid = false;
    float* pext_part = nullptr;     // [splits][K]
    int pext_splits = 0;
    // Gram form of the Newton path's output layer (tensor-core precisions, with G): one
    // stacked operand [G (Gt*128 rows) ; W_L rows of the cubature DOFs (Rt*128 rows)],
    // [rows][ldGs] in the precision's operand form (TF32-rounded FP32, or BF16 hi / lo).
    // Its G tiles give the row reductions over K (J^T M J = X_J^T G X_J, ...), its other
    // tiles the output rows the cubature reads.
    float* Gs32 = nullptr;
    __nv_bfloat16* Gsh = nullptr;
    __nv_bfloat16* Gsl = nullptr;
    int Gt = 0, Rt = 0, ldGs = 0, gs_rows_cap = 0;
    unsigned long long gs_G_mesh = 0;   // mesh id the G tiles were filled for
    int* cub_rows = nullptr;        // [gs_rows_cap] DOF of each cubature row (-1: none)
    float* Jc = nullptr;            // compact cubature rows [1 + r][Rt * 128]: u | J e_j
    size_t Jc_cap = 0;
    CUtensorMap tmGs[2];
    bool gs_ok = false;             // stacked operand ready (G part current)
    float* gy = nullptr;            // [K] G x_y, written by the G tiles' epilogue
    // the output stage's unfinished items (single-system Newton path): CTA c's item over
    // tile t in slot c * raw_m + (t - first tile of c), [128][Cp + 1] FP32 each; summed
    // and finished by k_out_finish
    float* out_part = nullptr;
    size_t out_part_cap = 0;
    int raw_m = 0;
    int row_part_cap = 0;           // rows of row_part (the finish kernel writes 4 per G tile)
    // weight network (cubature weights predicted at run time), first layer composed with
    // the output layer: h1 = sin(B1 x + c1), x the output layer's input (real column)
    int wn_H1 = 0, wn_H2 = 0, wn_H3 = 0, wn_ntet = 0;
    float* wn_B1 = nullptr;         // [H1][ldx] (ldx = the output layer's ld)
    float* wn_c1 = nullptr;         // [H1]
    float* wn_A2 = nullptr; float* wn_b2 = nullptr;   // [H2][H1], [H2]
    float* wn_A3 = nullptr; float* wn_b3 = nullptr;   // [H3][H2], [H3]
    float* wn_A4 = nullptr; float* wn_b4 = nullptr;   // [n_tet][H3], [n_tet]
    float* wn_h1 = nullptr;         // [2 kMaxWnetWidth] first-layer output | third-layer output
    float* wn_w = nullptr;          // [wn_cap] predicted weights of the cubature tets
    int wn_cap = 0;
    // linear subspace u = U p + (I - U U^T) D(q): U is stored as the first np rows of J
    float* V = nullptr;             // [ldK][np] W_L^T M U (filtered W_L; per mesh)
    float* UMU = nullptr;           // [np][np] U^T M U (per mesh)
    float* Uf = nullptr;            // [np] U^T f_ext (zero without f_ext)
    float* zpv = nullptr;           // [2 np] z_p = p - pbar - dt pbar_dot | p (per evaluation)
    float* lin_part = nullptr;      // [lin_blocks][np (1 + 2r)] partials of V^T X
    int lin_blocks = 0;
    unsigned long long V_mesh = 0;
};

}  // namespace dae

struct dae_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    std::string err;
    int* d_status = nullptr;         // device status word (first error wins)
    void* pinned = nullptr;          // host staging
    size_t pinned_bytes = 0;
    void* dstage = nullptr;          // device staging for host arguments
    size_t dstage_bytes = 0;
    int sm_count = 0;
    void* cublas = nullptr;          // cublasHandle_t (set-up GEMMs only)
    dae::NewtonState* last_ns = nullptr;   // state of the most recent newton step
    unsigned long long timeout_epoch = 0;  // bumped when the device reports DAE_ERR_TIMEOUT
    // instrumentation
    unsigned prof_on = 0;          // bit mask of instrumented phases
    long long launches = 0;             // kernels enqueued explicitly
    unsigned long long* d_kcount = nullptr;   // kernels executed inside graphs (device counter)
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    void* batch = nullptr;               // cached plan of dae_newton_step_batched
    void* batch_coupled = nullptr;       // cached plan of dae_newton_step_coupled
};

struct dae_decoder {
    dae_ctx* ctx = nullptr;
    int np = 0;                     // linear (PCA) basis size; the system has np + r unknowns
    unsigned long long id = 0;      // unique per upload and precision change
    int L = 0, r = 0, N = 0;
    std::vector<int> widths;
    dae_act act = DAE_ACT_TANH;
    dae_prec prec = DAE_FP32;
    std::vector<dae::Layer> layers;
    dae::Workspace ws;
    // work decomposition of the persistent layer chains, per hidden layer and direction
    // (0 forward, 1 reverse; layer order 0..L-2 in both): CTAs per 128-row tile as a K
    // split or as replicated K loops.  Empty: the fixed heuristic (chain_plan); set by
    // dae_decoder_autotune / dae_decoder_set_chain_plan for the precision in plan_prec.
    std::vector<int> plan_split[2], plan_rep[2];
    int plan_prec = -1;
    int cs_exact = 0;               // dae_eval_derivs with the exact multicomplex activation
};

struct dae_mesh {
    dae_ctx* ctx = nullptr;
    unsigned long long id = 0;      // unique per upload
    int n_vert = 0, n_tet = 0;
    dae_material material = DAE_STVK;
    double mu = 0, lam = 0;
    double* X = nullptr;       // [3V] rest positions
    int* tets = nullptr;       // [4T]
    float* Bm = nullptr;       // [T][9] Dm^{-1}, row-major
    float* vol = nullptr;      // [T] rest volumes
    float* mdof = nullptr;     // [3V] lumped mass per DOF
};

namespace dae {

// ----------------------------------------------------------------- kernels --
// Arguments shared by the forward epilogues.
struct FwdArgs {
    const float* W; int ld;                 // FP32 weights [m_pad][ld]
    const __nv_bfloat16* Wh; const __nv_bfloat16* Wl;
    const float* bias;
    const float* X; const __nv_bfloat16* Xh; const __nv_bfloat16* Xl;   // input [Cp][ld]
    int n_in, n_out, m_pad, r, Cp;
    int act;                                 // dae_act (hidden layers)
    int last;                                // 1: output layer
    int mode;                                // 0 forward hidden, 1 forward output,
                                             // 2 reverse (next g), 3 reverse (input layer)
    float* dout;                             // mode 3: delta_0 [1+r][r]
    // mode 1, fused row reductions (null row_part: not fused)
    float* row_part; int row_stride;         // per-tile [J^T a | Mr upper | B] partials
    const float* mdof; const float* f_ext; const float* zvec; double dt;
    float* a_out;                            // dense a_n (may be null)
    // hidden-layer outputs
    float* Y; __nv_bfloat16* Yh; __nv_bfloat16* Yl; int ldy;   // next activations [Cp][ldy]
    int out_bf16;                            // 0 none, 1 hi, 2 hi+lo
    int out_f32;                             // write FP32 activations (FP32 / TF32 inputs)
    const void* tmaps;                       // 4 CUtensorMap (tensor-core path)
    float* split_part;                       // split-K partial tiles [tiles][split][Cp][128]
    int* split_cnt;                          // per-tile arrival counters (kept at zero)
    float* S1; float* T;                     // reverse-pass data
    // output-layer outputs (any may be null)
    float* u; float* J; float* dJ; float* HDD; float* Hqq;
    double inv_h, inv_h2, inv_h3, inv_dt2;
    const NewtonState* ns;                   // early exit when ns->done (may be null)
    int* status;
    // mode 1 over the stacked Gram operand: tiles < gram_tiles are rows k < K of G X
    // (reductions into row_part, G x_y into gy); a later tile's row i is output row
    // row_map[i] (skipped when negative or i >= n_map)
    int gram_tiles, K;
    const int* row_map; int n_map;
    const float* Xg; int ldxg;               // FP32 input activations of the output layer [Cp][ldxg]
    const float* pext;                       // W_L^T f_ext [K] or null
    float* gy;                               // out: G x_y [K]
    // the cubature rows' u and J in compact form instead of at their DOFs (null: at the
    // DOFs): Jc[0][i] = u, Jc[1 + j][i] = J e_j for stacked row i < n_map, stride ldc
    float* Jc; int ldc;
    int exact;                               // 1: exact multicomplex columns (n_cols_exact)
};

// off: the decoder's coordinates start at entry off of the state (the linear subspace's
// np coordinates come first); qbar, qbar_dot point at the decoder's entries
void launch_seed(cudaStream_t s, const NewtonState* ns, const double* q_override,
                 const double* qbar, const double* qbar_dot, double dt, double h, int mode,
                 int r, int Cp, int ld0, float* X, __nv_bfloat16* Xh, __nv_bfloat16* Xl,
                 int out_bf16, float* zvec, int off = 0);
void launch_fwd_simt(cudaStream_t s, const FwdArgs& a);
// Input columns of the exact multicomplex batch (layout at n_cols_exact; modes as
// launch_seed).
void launch_seed_exact(cudaStream_t s, const double* q, const double* qbar, const double* qbar_dot,
                       double dt, double h, int mode, int r, int Cp, int ld0, float* X);
bool launch_fwd_tc(cudaStream_t s, const FwdArgs& a, dae_prec prec, int sm_count);

// Persistent layer-chain kernel (k_chain.cu): one job per GEMM layer.
// A layer of a chain is cut into tiles x P items (P = max(split, rep)): item (tile,
// ks) covers K chunk ks of `split` (split-K; the split CTAs of a tile exchange
// partial tiles and each finishes 128/split rows), or the whole K loop
// replicated `rep` times (short K; each copy finishes 128/rep rows).
struct ChainJob {
    CUtensorMap tm[4];           // A, A lo, B, B lo
    FwdArgs a;                   // epilogue (mode 0, 1, 2 or 3)
    int tiles, split, nk, rep;
    int cnt_off;                 // first per-tile arrival counter of this job (split > 1);
                                 // the chain zeroes a layer's counters once past it
    int stream;                  // 1: equal k-block ranges per CTA (output layer, mode 1)
    int item_base;               // grouped stage: position of this job's first tile in the
                                 // stage's item list (jobs of one stage are consecutive)
    int solo;                    // 1: every tile of the layer on CTA 0 (split = rep = 1); the
                                 // other CTAs skip the layer
    int raw;                     // stream job whose items are stored unfinished (raw_m slots
    int raw_m;                   // per CTA in the launch's split_part) for k_out_finish
    float* raw_part;             // raw job: the items' slots
    int rdy_off;                 // first per-tile ready counter of this layer (chains of one
                                 // decoder): arrivals of the CTAs finishing the tile's rows,
                                 // one counter per kRdyStride words (its own 128-byte line)
};
constexpr int kRdyStride = 32;
struct GridBar { unsigned count; unsigned gen; };
struct ChainLaunch {
    const ChainJob* jobs; int n_jobs; int Cp; int grid;
    GridBar* gb; const NewtonState* ns; int* status; float* split_part;
    unsigned* split_cnt;   // per-tile arrival counters of split layers (zero between launches)
    // Grouped launch (many decoders in one chain): stage t runs jobs
    // [stage_off[t], stage_off[t+1]) with no grid barrier between them, one item per
    // 128-row tile (no split, replication or streaming), and skips the jobs whose
    // a.ns is done.  stage_off == nullptr: one job per stage (a single decoder).
    const int* stage_off; int n_stages;
};
constexpr int kMaxGroupJobs = 512;   // jobs of one grouped stage
bool launch_chain(cudaStream_t s, const ChainLaunch& c, dae_prec prec);
// The output stage's raw items summed (in CTA order) and finished: G tiles' row
// reductions (kFinishBlocks partial rows per tile into a.row_part, G x_y), the cubature
// rows' u and J into a.Jc.  d_job: the stream job (device copy, `tiles` tiles, Cp
// columns) whose launch over `grid` CTAs stored them in `part`.
void launch_out_finish(cudaStream_t s, const ChainJob* d_job, int tiles, int Cp, const float* part,
                       int grid, const NewtonState* ns);
constexpr int kFinishRows = 32;                   // rows per block of k_out_finish
constexpr int kFinishBlocks = 128 / kFinishRows;  // blocks (partial rows) per tile
void launch_store_job(cudaStream_t s, ChainJob* dst, const ChainJob& job);
int run_wait_selftest(cudaStream_t s, GridBar* gb, int* out, int nblocks);
// Work decomposition of one chain layer: sets job.split and job.rep.
void chain_plan(ChainJob& job, int grid);
constexpr int kMaxSplit = 16;
int tc_split(int m_pad, int ld, dae_prec prec, int sm_count);

struct RowArgs {
    const float* J; const float* dJ; const float* HDD; const float* mdof; const float* f_ext;
    const float* zvec; float* a; float* part; int N, r, stride; double dt;
    const NewtonState* ns;
};
void launch_row_reduce(cudaStream_t s, const RowArgs& a, int n_blocks);

struct CubArgs {
    int w_stride;                            // weights per frame (cub_w + frame * w_stride)
    const float* u; const float* J; int N, r;
    const double* X; const int* tets; const float* Bm; const float* vol; int n_tet;
    int material; float mu, lam;
    const int* cub_tets; const float* cub_w; int n_cub;
    float* fe_w; int* fe_dof; float* part; double* energy; int stride;
    const NewtonState* ns; int* eval_flag;   // set when a Neo-Hookean tet is inverted
    // linear subspace: u += U p at the tet's DOFs (U = the first np rows of J, p = pv)
    int np; const float* pv;
    // compact cubature rows written by the output stage (null: read u and J at the DOFs):
    // [1 + r - np][ldc], row 12 slot + 3 a + d, column 0 = u, column 1 + j = J e_j
    const float* Jc; int ldc;
    int n_parts;                             // partial rows (blocks): cubature_parts(n_cub)
};
void launch_cubature(cudaStream_t s, const CubArgs& a);
// partial rows of the cubature kernel for n_cub tets (one per block)
int cubature_parts(int n_cub, int sm_count);

struct WtaArgs {
    const float* W; int ld, N, K;           // dense matrix [N][ld] (W_L, or G with N = K)
    const float* a;                          // dense seed [N]
    const float* Wp; int ldp;                // matrix of the cubature pair rows (W_L)
    const float* pext; float pext_scale;     // extra split: pext_scale * pext (or null)
    const float* gy;                         // extra split: gy (or null), after pext
    const int* run_flag;                     // skip when *run_flag == 0 (or null)
    const float* fe_w; const int* fe_dof; int n_pairs; double dt2;
    float* part; int nsplit_dense, nsplit_pairs;   // out [nsplit_dense + nsplit_pairs][K]
    const NewtonState* ns;
};
void launch_wta(cudaStream_t s, const WtaArgs& a);
void launch_xy(cudaStream_t s, const float* X, int ld, int K, int r, const float* zvec, double h,
               float* xy, const NewtonState* ns);
void launch_scale_rows(cudaStream_t s, const float* W, int ld, const float* m, int rows, float* out);
void launch_fext_check(cudaStream_t s, const float* f, const float* prev, int N, int* flag);
void launch_pext_finish(cudaStream_t s, const float* part, int splits, int K, float* pext,
                        const float* f, float* prev, int N, int* flag);

struct BwdArgs {
    const float* W; int ld;                  // layer weights [m_pad][ld], rows = n_o, cols = n_i
    int n_o, n_i, r;
    const float* in_part; int in_split; int in_ncol;  // incoming delta partials [in_split][in_ncol][n_o]
    const float* S1; const float* T;         // layer derivative data
    float* g;                                // scratch [1+r][n_o]
    float* out_part; int out_split;          // [out_split][1+r][n_i]
    const NewtonState* ns;
};
void launch_bwd(cudaStream_t s, const BwdArgs& a);
// g of the top hidden layer in the tensor-core B layout [Cb][ld] (FP32 and/or BF16 splits)
void launch_bwd_prep_tc(cudaStream_t s, const BwdArgs& a, int Cb, int ld, float* g32,
                        __nv_bfloat16* gh, __nv_bfloat16* gl, int out_f32, int out_bf16);
void launch_transpose(cudaStream_t s, const float* W, int ld, int rows, int cols, float* WT, int ldT);
int bwd_split(int n_i, int n_o, int sm);

struct AsmArgs {
    int r; double dt, h;
    const float* row_part; int n_row_blocks, row_stride;
    const float* cub_part; const double* cub_energy; int n_cub, cub_stride;
    int cub_parts;                           // partial rows of the cubature kernel
    const float* bwd_part; int bwd_split;   // [split][1+r][r]
    double* red;                             // out: phi | A | energy | terms
    NewtonState* ns;                         // null: assemble only
    int control;                             // 1: Newton control step
    double tol, c_armijo, max_step, xtol; int max_iter, max_halvings, max_evals;
    int* eval_flag;                          // per-evaluation flag of the cubature kernel
    int* status;                             // sticky device status (assemble-only mode)
    float* lu;                               // stored FP32 Newton-matrix factors (control)
    cudaGraphConditionalHandle hcond; int use_cond;
    unsigned long long* kcount; int kpe;
    // linear subspace (np > 0): r above is the system size np + rq
    int rq, np;
    const float* lin_part; int lin_blocks;   // V^T X partials
    const float* UMU; const float* Uf;
    const double* qbar; const double* qbar_dot;   // full state arrays
    const double* q_in;                      // evaluation point when ns is null
};
// One evaluation's FP64 end in two launches around the reverse pass:
//   launch_decide   column sums of the row, cubature and linear-subspace partials and the
//                   energy, then phi (Eq. 10) and, under Newton control, the line-search
//                   decision (k_decide); a trial that is not accepted for a new Newton step
//                   sets ns->skip_rev, which every reverse-pass kernel honours
//   launch_control  the Newton matrix A (Eq. 11) from the reverse-pass partials and the
//                   sums above, the solve A delta = -phi and the next trial (k_control)
void launch_decide(cudaStream_t s, const AsmArgs& a);
void launch_control(cudaStream_t s, const AsmArgs& a);
// true when the reverse pass of this evaluation is skipped (device side)
__device__ __forceinline__ bool skip_reverse(const NewtonState* ns) {
    return ns && (ns->done || ns->skip_rev);
}

// ------------------------------------------------ grouped (batched) launches --
// The kernels of one Newton evaluation run for many independent systems (decoder +
// mesh + Newton state each) in one launch: blockIdx.z selects the system's argument
// record in a device array; a system whose Newton state is done returns at once.
struct CtlArgs {
    cudaGraphConditionalHandle hcond; int use_cond;   // evaluation loop of a graph frame
    unsigned long long* kcount; int kpe;              // executed-kernel counter
    int r; double dt, h;
    const double* rowsum; const double* cubsum; const double* esum;
    const float* bwd_part; int bwd_split;             // reverse-pass partials [split][(1+rq) rq]
    int have_cub;
    double* red;
    NewtonState* ns; int control;
    double tol, c_armijo, max_step, xtol; int max_iter, max_halvings, max_evals;
    int* eval_flag;     // set by the cubature kernel (inverted tet) for this evaluation
    int* status;
    float* lu;          // FP32 factors of the last Newton matrix (null: no step estimate)
    int rq, np;                              // decoder latent size, linear basis size (r = np + rq)
    const double* linsum;                    // [np][1 + 2 rq] sums of V^T X
    const float* UMU; const float* Uf;
    const double* qbar; const double* qbar_dot; const double* q_in;
};
struct SeedArgs {
    const NewtonState* ns; const double* qbar; const double* qbar_dot; double dt, h;
    int r, Cp, ld0; float* X; __nv_bfloat16* Xh; __nv_bfloat16* Xl; int out_bf16; float* zvec;
    int off;   // first state entry of the decoder's coordinates (linear subspace size)
};
struct XyArgs {
    const float* X; int ld, K, r; const float* zvec; double h; float* xy; const NewtonState* ns;
};
struct PrepArgs {
    BwdArgs a; int Cb, ld; float* g32; __nv_bfloat16* gh; __nv_bfloat16* gl; int out_f32, out_bf16;
};
struct ColsumArgs {
    const float* part; int n_parts, stride, n_ent; double* out; const NewtonState* ns;
};
struct DsumArgs { const double* x; int n; double* out; const NewtonState* ns; };
struct FrameArgs {
    NewtonState* ns; const double* q0; double* q_out; int r;
};
// The three column sums, the energy sum and the control step of launch_assemble.
void assemble_parts(const AsmArgs& a, ColsumArgs cs[4], DsumArgs& ds, CtlArgs& c);
void launch_seed_batched(cudaStream_t s, const SeedArgs* d_args, int n_sys, int max_elems);
void launch_cubature_batched(cudaStream_t s, const CubArgs* d_args, int n_sys, int max_parts);
void launch_xy_batched(cudaStream_t s, const XyArgs* d_args, int n_sys, int max_K);
void launch_wta_batched(cudaStream_t s, const WtaArgs* d_args, int n_sys, int max_K, int max_splits);
void launch_bwd_prep_tc_batched(cudaStream_t s, const PrepArgs* d_args, int n_sys, int max_ld);
void launch_decide_batched(cudaStream_t s, const ColsumArgs* cs, const DsumArgs* ds,
                           const CtlArgs* c, int n_sys, int max_ent);
void launch_control_batched(cudaStream_t s, const CtlArgs* c, int n_sys);
void launch_frame_begin_batched(cudaStream_t s, const FrameArgs* f, int n_sys,
                                cudaGraphConditionalHandle h, int use);
void launch_frame_end_batched(cudaStream_t s, const FrameArgs* f, int n_sys);
// sets the graph condition h (flag == nullptr) or writes *flag: 1 while any system runs
void launch_batch_cond(cudaStream_t s, const FrameArgs* f, int n_sys, cudaGraphConditionalHandle h,
                       int* flag);
// Weight network: h1 = sin(B1 x + c1) (x = real column of the output layer's input,
// stride 1), h2 = sin(A2 h1 + b2), h3 = sin(A3 h2 + b3), w_j = (A4[tets[j]] h3 + b4[tets[j]])^2.
// With ns: skipped once the frame is done, and after its first evaluation when
// first_only (the weights hold for the frame).
constexpr int kMaxWnetWidth = 1024;   // hidden widths of the weight network
struct WnetArgs {
    const float* x; int K; int ldx;
    const float* B1; const float* c1; int H1;
    const float* A2; const float* b2; int H2;
    const float* A3; const float* b3; int H3;
    const float* A4; const float* b4;
    const int* tets; int n; float* h1; float* w;
    const NewtonState* ns; int first_only;
};
void launch_wnet(cudaStream_t s, const WnetArgs& a);
void launch_wnet_batched(cudaStream_t s, const WnetArgs* d_args, int n_sys, int max_H1, int max_n);
// Linear-subspace terms of one evaluation: part[b][a][c] = sum over the 128 rows k of block
// b of V[k][a] X_c[k] for the columns c = 3 (H[D,D]), kShared+3j (J), kShared+3j+2 (dJ);
// vz[k] = (V z_p)[k] (a reverse-pass seed split: W_L^T M U z_p); block 0 also writes
// zpv = [z_p | p] (from ns->q_trial or q_in, and the full qbar / qbar_dot).
struct LinArgs {
    const float* X; int K, ldx, r, np;
    const float* V; float* part; float* vz; float* zpv;
    const NewtonState* ns; const double* q_in; const double* qbar; const double* qbar_dot; double dt;
};
void launch_linear(cudaStream_t s, const LinArgs& a, int n_blocks);
// grouped form (z = system; systems without a linear subspace have np = 0)
void launch_linear_batched(cudaStream_t s, const LinArgs* d_args, int n_sys, int max_blocks);
// ------------------------------------------------------ coupled domains --
// Domains of a substructured body tied at interface vertices (penalty springs of
// stiffness k_c between vertices that coincide at rest, and anchors holding a vertex at
// rest; deformation substructuring, Sec. 6), stepped as one Newton system over all
// domains' latents.  A tie vertex t is one (domain, vertex) that takes part in a tie.
struct TieDom {
    const float* X; int ldx;        // FP32 input activations of the output layer [Cp][ldx]
    const float* W; int ld;         // output layer FP32 weights [m_pad][ld]
    const float* b;                 // output layer bias
    int K, r, off;                  // hidden width, latent size, first global unknown
    NewtonState* ns;                // the domain's Newton state (q slices, flags)
    const double* red;              // the domain's phi | A | energy buffer
    float* fe_w; int* fe_dof;       // reverse-pass seed pairs; the tie forces go to [pair0, ...)
    int pair0;                      // 12 n_cub
    int* eval_flag;                 // cubature flag of the domain's evaluation
};
struct CoupledState {
    double merit_acc, phi_norm0, alpha, energy, coupling_energy;
    int halvings, iters, evals, done, converged, status, nfull, skip;
};
struct CoupledArgs {
    int n_dom, n_tv, n_tot;
    const TieDom* dom;
    const int* unk_dom;                    // domain of global unknown k
    const int* dtv_off; const int* dtv;    // CSR: tie vertices of domain d
    const int* tv_dom; const int* tv_vert; const int* tv_slot;   // per tie vertex
    const int* nb_off; const int* nb;      // CSR: tie vertices paired with tie vertex t
    const int* n_anch;                     // anchors at tie vertex t
    float* uJ;                             // [n_tv][3][1 + kMaxR]: u and J at the 3 DOFs
    double* g;                             // [n_tv][3] tie force dE_c/du
    double kc, dt, h;
    CoupledState* cs;
    double* q_acc; double* q_trial; double* delta; double* phi;   // [n_tot]
    double tol, c_armijo, max_step, xtol; int max_iter, max_halvings, max_evals;
    // block solve over the domain forest: components, domains in post-order (children
    // before parents), parents (-1: a component's root), the pairs of a child with its
    // parent (tie vertex of the child, of the parent)
    int n_comp; const int* comp_off; const int* order; const int* parent;
    const int* cp_off; const int* cp;      // CSR over child domains: 2 ints per pair
    double* S; double* X; double* y; int* piv;   // per domain [32 * 32], [32 * 32], [32], [32]
};
void launch_tie_uj(cudaStream_t s, const CoupledArgs* d_args, int n_tv);
void launch_coupled_decide(cudaStream_t s, const CoupledArgs* d_args);
void launch_coupled_solve(cudaStream_t s, const CoupledArgs* d_args, int n_comp);
void launch_coupled_update(cudaStream_t s, const CoupledArgs* d_args);
void launch_coupled_begin(cudaStream_t s, const CoupledArgs* d_args);
// copy[i]: n bytes from src to dst (device memory), one block per copy
struct CopyDesc { const void* src; void* dst; unsigned long long n; };
void launch_copy_batch(cudaStream_t s, const CopyDesc* d, int n);
// doubles of the reduced-system buffer: outputs, terms and reduction scratch
inline size_t red_size(int r) {
    size_t nsym = (size_t)r * (r + 1) / 2;
    return (size_t)r + r * r + 1 + 4 * (size_t)r * r + r + (r + nsym + (size_t)r * r) + (r + nsym) +
           (size_t)(1 + r) * r + 1 + (size_t)r * (1 + 2 * r);
}

void launch_roll_setup(cudaStream_t s, RollCtl* rc, int n_frames, int given_q0, int advance,
                       const double* q_in, int r);
void launch_roll_init(cudaStream_t s, RollCtl* rc, cudaGraphConditionalHandle h, int use,
                      unsigned long long* kcount);
void launch_frame_start(cudaStream_t s, RollCtl* rc, NewtonState* ns, const double* qbar,
                        const double* qbar_dot, double dt, int r, cudaGraphConditionalHandle h,
                        int use, unsigned long long* kcount);
void launch_frame_finish(cudaStream_t s, RollCtl* rc, NewtonState* ns, double* qbar,
                         double* qbar_dot, double dt, int r, double* traj, NewtonState* hist,
                         double* q_out, cudaGraphConditionalHandle h, int use,
                         unsigned long long* kcount);
bool make_tmap(void* out, const void* base, bool fp32, int ld, int rows, int box_rows);
void launch_split_bf16(cudaStream_t s, const float* W, __nv_bfloat16* hi, __nv_bfloat16* lo,
                       size_t n);
void launch_round_tf32(cudaStream_t s, const float* W, float* out, size_t n);
// Rows of the stacked Gram operand for the cubature DOFs: row i < 12 n_cub is output-layer
// row dof(i) = 3 tets[4 cub_tets[i/12] + (i%12)/3] + i%3 (the order of the element
// force pairs), copied from the output layer's operand arrays (src32 or srch/srcl,
// [*][ld]) into dst rows [row0 + i]; rows i in [12 n_cub, n_rows) are zeroed; map[i] = dof
// or -1.
struct GatherArgs {
    const int* cub_tets; const int* tets; int n_cub, n_rows, ld, row0;
    const float* src32; const __nv_bfloat16* srch; const __nv_bfloat16* srcl;
    float* dst32; __nv_bfloat16* dsth; __nv_bfloat16* dstl; int* map;
};
void launch_gather_cub_rows(cudaStream_t s, const GatherArgs* d_args, const GatherArgs& host_args,
                            int n_sys);

}  // namespace dae
