// Internal declarations of the decoder training pass (k_train.cu, train.cu).
#pragma once
#include "dae_internal.h"

namespace dae {

// One GEMM operand in the two layouts the training GEMMs read, as split BF16 hi/lo:
// planes [c][k] (row stride ldc, K = neurons contiguous) and rows [k][c] (row stride
// ldn, K = batch columns contiguous).
// In the FP32 form the operands are FP32 copies in the same two layouts (cf, nf; the
// BF16 arrays are then unused).
struct Operand {
    __nv_bfloat16* ch; __nv_bfloat16* cl; int ldc;
    __nv_bfloat16* nh; __nv_bfloat16* nl; int ldn;
    float* cf; float* nf;
};

// D[M][N] = A[M][K] B[N][K]^T (split BF16x3, FP32 accumulation), tensor maps of the
// K-major A hi, A lo, B hi, B lo (64-element boxes of 128 rows).
struct GemmArgs {
    CUtensorMap tm[4];
    float* out; int ldo;
    int out_mode;            // 0: out[m * ldo + n];  1: out[n * ldo + m]
    int M, N;                // stored extent
    int nk;                  // K blocks of 64 elements
    const float* bias; int bias_cols;   // out += bias[m] for n < bias_cols (mode 1)
    int* status;
    // FP32 form: the same product from FP32 operands A [M][lda], B [N][ldb] (K-major, K
    // padded to nk 64-element blocks with zeros in A or B)
    const float* a32; int lda; const float* b32; int ldb;
};

bool launch_gemm_x3(cudaStream_t s, const GemmArgs& g, int m_tiles, int n_tiles);
// D = A B^T in FP32 on the CUDA cores (FFMA, FP32 accumulation), 64 x 64 tiles.
bool launch_gemm_f32(cudaStream_t s, const GemmArgs& g);
// FP32 padded copies of W ([m_pad][ld]) and W^T ([n_pad][ldT], when wt is not null).
void launch_train_weights_f32(cudaStream_t s, const float* W, int n_out, int n_in, float* w, int ld,
                              float* wt, int ldT);
void launch_train_seed(cudaStream_t s, const double* q, int B, int r, const Operand& X);
void launch_train_act(cudaStream_t s, const float* Z, int ldz, int n, int B, int r, int act,
                      const Operand& X);
void launch_train_act_bwd(cudaStream_t s, const float* Xb, int ldx, const float* Z, int ldz, int n,
                          int B, int r, int act, const Operand& Zb, float* zb_val);
void launch_train_split(cudaStream_t s, const float* g, int n, int B, int r, const Operand& Zb);
void launch_train_bias_grad(cudaStream_t s, const float* zb_val, int ld, int n, int B, float* gb);
void launch_train_grad_q(cudaStream_t s, const float* zb_val, int n1, const float* W1, int ldw, int B,
                         int r, double* gq);
void launch_train_weights(cudaStream_t s, const float* W, int n_out, int n_in, __nv_bfloat16* h,
                          __nv_bfloat16* l, int ld, __nv_bfloat16* th, __nv_bfloat16* tl, int ldT);

}  // namespace dae
