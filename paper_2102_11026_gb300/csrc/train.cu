// Host side of the decoder training pass (C ABI dae_trainer_*, dae_train_*): the
// batched first-order forward of u = D(q), J = dD/dq and its reverse sweep, with the
// forward activations checkpointed every second layer and recomputed in between.
#include <algorithm>
#include <cstring>
#include <vector>
#include "train_internal.h"

using namespace dae;

struct dae_trainer {
    dae_ctx* ctx = nullptr;
    int L = 0, r = 0, Bmax = 0, Cpad = 0, last_B = -1;
    dae_act act = DAE_ACT_TANH;
    std::vector<int> widths;
    struct TL {
        int n_in, n_out, ld, m_pad, ldT, mT_pad;
        __nv_bfloat16 *wh = nullptr, *wl = nullptr, *wth = nullptr, *wtl = nullptr;
        float *wf = nullptr, *wtf = nullptr;       // FP32 form: padded W and W^T
        CUtensorMap tmW[2], tmWT[2];
    };
    dae_prec prec = DAE_BF16X3;   // GEMM arithmetic: split BF16x3 (tensor cores) or FP32
    float* opf[3][2] = {};        // FP32 operand arrays (planes, rows) of X[0], X[1], Zb
    std::vector<TL> layers;
    Operand X[2] = {};            // activations of a layer boundary (ping-pong)
    Operand Zb = {};              // cotangent of a layer's pre-activation
    CUtensorMap tmXc[2][2], tmXn[2][2], tmZc[2], tmZn[2];
    int ldx = 0, nx_pad = 0, ldz = 0, nz_pad = 0, nmax = 0;
    std::vector<float*> Zck;      // FP32 pre-activations [Cpad][ldz] of the even hidden boundaries
    float* Ztmp = nullptr;        // a recomputed odd boundary
    float* Xbar = nullptr;        // FP32 [Cpad][ldz] reverse-pass output before the activation
    float* zval = nullptr;        // FP32 [Bmax][nmax] value rows of the current cotangent
};

namespace {

size_t rup(size_t x, size_t m) { return (x + m - 1) / m * m; }

dae_status tfail(dae_ctx* ctx, dae_status st, const char* msg) {
    if (ctx) ctx->err = msg;
    return st;
}

#define TCU(ctx, x)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess) return tfail((ctx), DAE_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
dae_status talloc(dae_ctx* ctx, T** p, size_t n) {
    *p = nullptr;
    if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return tfail(ctx, DAE_ERR_OOM, "device allocation failed (trainer)");
    }
    TCU(ctx, cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T)));
    return DAE_OK;
}

#define TTRY(x)                         \
    do {                                \
        dae_status s_ = (x);            \
        if (s_ != DAE_OK) return s_;    \
    } while (0)

bool on_dev(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

dae_status alloc_operand(dae_trainer* t, Operand& P, int ldc, int nrows) {
    dae_ctx* ctx = t->ctx;
    P.ldc = ldc;
    P.ldn = t->Cpad;
    TTRY(talloc(ctx, &P.ch, (size_t)t->Cpad * ldc));
    TTRY(talloc(ctx, &P.cl, (size_t)t->Cpad * ldc));
    TTRY(talloc(ctx, &P.nh, (size_t)nrows * t->Cpad));
    TTRY(talloc(ctx, &P.nl, (size_t)nrows * t->Cpad));
    return DAE_OK;
}

void free_operand(Operand& P) {
    cudaFree(P.ch); cudaFree(P.cl); cudaFree(P.nh); cudaFree(P.nl);
    P = Operand{};
}

// D = A B^T with A, B given as tensor maps (split BF16x3) and as FP32 arrays (FP32 form).
GemmArgs gemm(const CUtensorMap* a, const float* a32, int lda, const CUtensorMap* b, const float* b32,
              int ldb, float* out, int ldo, int mode, int M, int N, int nk, const float* bias,
              int bias_cols, int* status) {
    GemmArgs g;
    memset(&g, 0, sizeof g);
    g.tm[0] = a[0]; g.tm[1] = a[1]; g.tm[2] = b[0]; g.tm[3] = b[1];
    g.out = out; g.ldo = ldo; g.out_mode = mode; g.M = M; g.N = N; g.nk = nk;
    g.bias = bias; g.bias_cols = bias_cols; g.status = status;
    g.a32 = a32; g.lda = lda; g.b32 = b32; g.ldb = ldb;
    return g;
}

dae_status run_gemm(dae_trainer* t, const GemmArgs& g) {
    dae_ctx* ctx = t->ctx;
    ctx->launches += 1;
    const bool ok = t->prec == DAE_FP32 ? launch_gemm_f32(ctx->stream, g)
                                        : launch_gemm_x3(ctx->stream, g, (g.M + 127) / 128, (g.N + 127) / 128);
    if (!ok) return tfail(ctx, DAE_ERR_CUDA, "training GEMM launch failed");
    return DAE_OK;
}

dae_status check_args(dae_trainer* t, const float* const* W, const float* const* b, int B,
                      const double* q) {
    dae_ctx* ctx = t ? t->ctx : nullptr;
    if (!t || !W || !b || !q) return tfail(ctx, DAE_ERR_INVALID_ARG, "trainer, weights or latents missing");
    if (B < 1 || B > t->Bmax) return tfail(ctx, DAE_ERR_INVALID_ARG, "batch outside 1..max_batch");
    for (int l = 0; l < t->L; ++l)
        if (!W[l] || !b[l] || !on_dev(W[l]) || !on_dev(b[l]))
            return tfail(ctx, DAE_ERR_INVALID_ARG, "trainer weights must be device arrays");
    if (!on_dev(q)) return tfail(ctx, DAE_ERR_INVALID_ARG, "trainer latents must be a device array");
    TCU(ctx, cudaSetDevice(ctx->device));
    return DAE_OK;
}

// Weights of every layer as split BF16 (and their transposes when `transposed`).
void stage_weights(dae_trainer* t, const float* const* W, bool transposed) {
    for (int l = 0; l < t->L; ++l) {
        auto& y = t->layers[l];
        t->ctx->launches += 1;
        if (t->prec == DAE_FP32)
            launch_train_weights_f32(t->ctx->stream, W[l], y.n_out, y.n_in, y.wf, y.ld,
                                     transposed ? y.wtf : nullptr, y.ldT);
        else
            launch_train_weights(t->ctx->stream, W[l], y.n_out, y.n_in, y.wh, y.wl,  y.ld,
                                 transposed ? y.wth : nullptr, transposed ? y.wtl : nullptr, y.ldT);
    }
}

// New batch size: the batch columns past C = B (1 + r) of the row-layout operands are
// contracted over by the weight-gradient GEMMs and must be zero.
dae_status set_batch(dae_trainer* t, int B) {
    if (B == t->last_B) return DAE_OK;
    dae_ctx* ctx = t->ctx;
    for (Operand* P : {&t->X[0], &t->X[1], &t->Zb}) {
        const size_t n = (size_t)P->ldn * (P == &t->Zb ? t->nz_pad : t->nx_pad);
        TCU(ctx, cudaMemsetAsync(P->nh, 0, n * sizeof(__nv_bfloat16), ctx->stream));
        TCU(ctx, cudaMemsetAsync(P->nl, 0, n * sizeof(__nv_bfloat16), ctx->stream));
        if (P->nf) TCU(ctx, cudaMemsetAsync(P->nf, 0, n * sizeof(float), ctx->stream));
    }
    t->last_B = B;
    return DAE_OK;
}

// Z_l = W_l X_{l-1} + b_l on the value columns, X_{l-1} in ping-pong buffer (l-1)&1.
dae_status forward_layer(dae_trainer* t, int l, const float* bias, int B, float* out, int ldo) {
    auto& y = t->layers[l - 1];
    const int C = B * (1 + t->r);
    const int xb = (l - 1) & 1;
    return run_gemm(t, gemm(y.tmW, y.wf, y.ld, t->tmXc[xb], t->X[xb].cf, t->X[xb].ldc, out, ldo, 1,
                            y.n_out, C, y.ld / 64, bias, B, t->ctx->d_status));
}

}  // namespace

extern "C" {

dae_status dae_trainer_create(dae_ctx* ctx, int n_layers, const int* widths, dae_act act,
                              int max_batch, dae_trainer** out) {
    if (!ctx || !widths || !out || n_layers < 1 || max_batch < 1)
        return tfail(ctx, DAE_ERR_INVALID_ARG, "trainer: bad arguments");
    *out = nullptr;
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 1) return tfail(ctx, DAE_ERR_INVALID_ARG, "trainer: widths must be positive");
    if (widths[0] > kMaxR) return tfail(ctx, DAE_ERR_UNSUPPORTED, "trainer: latent size above 32");
    TCU(ctx, cudaSetDevice(ctx->device));
    dae_trainer* t = new dae_trainer();
    t->ctx = ctx;
    t->L = n_layers;
    t->r = widths[0];
    t->Bmax = max_batch;
    t->act = act;
    t->widths.assign(widths, widths + n_layers + 1);
    t->Cpad = (int)rup((size_t)max_batch * (1 + t->r), 128);
    auto cleanup = [&](dae_status st) { dae_trainer_free(t); return st; };
    int wx = 1, wz = 1;
    for (int l = 0; l < n_layers; ++l) wx = std::max(wx, widths[l]);          // activation widths
    for (int l = 1; l <= n_layers; ++l) wz = std::max(wz, widths[l]);         // pre-activation widths
    t->ldx = (int)rup(wx, 64);
    t->nx_pad = (int)rup(wx, 128);
    t->ldz = (int)rup(std::max(wz, wx), 64);
    t->nz_pad = (int)rup(wz, 128);
    t->nmax = std::max(wx, wz);
    t->layers.resize(n_layers);
    for (int l = 0; l < n_layers; ++l) {
        auto& y = t->layers[l];
        y.n_in = widths[l];
        y.n_out = widths[l + 1];
        y.ld = (int)rup(y.n_in, 64);
        y.m_pad = (int)rup(y.n_out, 128);
        y.ldT = (int)rup(y.n_out, 64);
        y.mT_pad = (int)rup(y.n_in, 128);
        dae_status st;
        if ((st = talloc(ctx, &y.wh, (size_t)y.m_pad * y.ld)) || (st = talloc(ctx, &y.wl, (size_t)y.m_pad * y.ld)) ||
            (st = talloc(ctx, &y.wth, (size_t)y.mT_pad * y.ldT)) ||
            (st = talloc(ctx, &y.wtl, (size_t)y.mT_pad * y.ldT)))
            return cleanup(st);
        bool ok = make_tmap(&y.tmW[0], y.wh, false, y.ld, y.m_pad, 128) &&
                  make_tmap(&y.tmW[1], y.wl, false, y.ld, y.m_pad, 128) &&
                  make_tmap(&y.tmWT[0], y.wth, false, y.ldT, y.mT_pad, 128) &&
                  make_tmap(&y.tmWT[1], y.wtl, false, y.ldT, y.mT_pad, 128);
        if (!ok) return cleanup(tfail(ctx, DAE_ERR_UNSUPPORTED, "trainer: tensor map encoding failed"));
    }
    dae_status st;
    for (int i = 0; i < 2; ++i)
        if ((st = alloc_operand(t, t->X[i], t->ldx, t->nx_pad))) return cleanup(st);
    if ((st = alloc_operand(t, t->Zb, t->ldz, t->nz_pad))) return cleanup(st);
    for (int i = 0; i < 2; ++i) {
        bool ok = make_tmap(&t->tmXc[i][0], t->X[i].ch, false, t->ldx, t->Cpad, 128) &&
                  make_tmap(&t->tmXc[i][1], t->X[i].cl, false, t->ldx, t->Cpad, 128) &&
                  make_tmap(&t->tmXn[i][0], t->X[i].nh, false, t->Cpad, t->nx_pad, 128) &&
                  make_tmap(&t->tmXn[i][1], t->X[i].nl, false, t->Cpad, t->nx_pad, 128);
        if (!ok) return cleanup(tfail(ctx, DAE_ERR_UNSUPPORTED, "trainer: tensor map encoding failed"));
    }
    bool ok = make_tmap(&t->tmZc[0], t->Zb.ch, false, t->ldz, t->Cpad, 128) &&
              make_tmap(&t->tmZc[1], t->Zb.cl, false, t->ldz, t->Cpad, 128) &&
              make_tmap(&t->tmZn[0], t->Zb.nh, false, t->Cpad, t->nz_pad, 128) &&
              make_tmap(&t->tmZn[1], t->Zb.nl, false, t->Cpad, t->nz_pad, 128);
    if (!ok) return cleanup(tfail(ctx, DAE_ERR_UNSUPPORTED, "trainer: tensor map encoding failed"));
    t->Zck.assign(n_layers, nullptr);
    for (int k = 2; k < n_layers; k += 2)
        if ((st = talloc(ctx, &t->Zck[k], (size_t)t->Cpad * t->ldz))) return cleanup(st);
    if ((st = talloc(ctx, &t->Ztmp, (size_t)t->Cpad * t->ldz)) ||
        (st = talloc(ctx, &t->Xbar, (size_t)t->Cpad * t->ldz)) ||
        (st = talloc(ctx, &t->zval, (size_t)max_batch * t->nmax)))
        return cleanup(st);
    *out = t;
    return DAE_OK;
}

dae_status dae_trainer_free(dae_trainer* t) {
    if (!t) return DAE_ERR_INVALID_ARG;
    cudaSetDevice(t->ctx->device);
    cudaStreamSynchronize(t->ctx->stream);
    for (auto& y : t->layers) {
        cudaFree(y.wh); cudaFree(y.wl); cudaFree(y.wth); cudaFree(y.wtl); cudaFree(y.wf); cudaFree(y.wtf);
    }
    for (auto& pr : t->opf) { cudaFree(pr[0]); cudaFree(pr[1]); }
    free_operand(t->X[0]);
    free_operand(t->X[1]);
    free_operand(t->Zb);
    for (auto p : t->Zck) cudaFree(p);
    cudaFree(t->Ztmp); cudaFree(t->Xbar); cudaFree(t->zval);
    delete t;
    return DAE_OK;
}

dae_status dae_trainer_set_precision(dae_trainer* t, dae_prec prec) {
    if (!t) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = t->ctx;
    if (prec != DAE_FP32 && prec != DAE_BF16X3)
        return tfail(ctx, DAE_ERR_UNSUPPORTED, "trainer: FP32 or BF16X3 only");
    TCU(ctx, cudaSetDevice(ctx->device));
    TCU(ctx, cudaStreamSynchronize(ctx->stream));
    if (prec == DAE_FP32 && !t->opf[0][0]) {
        // FP32 operands in both layouts and padded FP32 weights (zeroed once: padding)
        Operand* ops[3] = {&t->X[0], &t->X[1], &t->Zb};
        const int nrows[3] = {t->nx_pad, t->nx_pad, t->nz_pad};
        for (int i = 0; i < 3; ++i) {
            TTRY(talloc(ctx, &t->opf[i][0], (size_t)t->Cpad * ops[i]->ldc));
            TTRY(talloc(ctx, &t->opf[i][1], (size_t)nrows[i] * t->Cpad));
        }
        for (auto& y : t->layers) {
            TTRY(talloc(ctx, &y.wf, (size_t)y.m_pad * y.ld));
            TTRY(talloc(ctx, &y.wtf, (size_t)y.mT_pad * y.ldT));
        }
    }
    Operand* ops[3] = {&t->X[0], &t->X[1], &t->Zb};
    for (int i = 0; i < 3; ++i) {
        ops[i]->cf = prec == DAE_FP32 ? t->opf[i][0] : nullptr;
        ops[i]->nf = prec == DAE_FP32 ? t->opf[i][1] : nullptr;
    }
    t->prec = prec;
    t->last_B = -1;   // the row layouts' padding is zeroed again for the new form
    return DAE_OK;
}

dae_status dae_train_forward(dae_trainer* t, const float* const* W, const float* const* b, int B,
                             const double* q, float* uJ) {
    TTRY(check_args(t, W, b, B, q));
    dae_ctx* ctx = t->ctx;
    if (!uJ || !on_dev(uJ)) return tfail(ctx, DAE_ERR_INVALID_ARG, "uJ must be a device array");
    cudaStream_t s = ctx->stream;
    const int L = t->L, r = t->r, C = B * (1 + r);
    TTRY(set_batch(t, B));
    stage_weights(t, W, false);
    ctx->launches += 1;
    launch_train_seed(s, q, B, r, t->X[0]);
    for (int l = 1; l <= L; ++l) {
        if (l == L) {
            TTRY(forward_layer(t, l, b[l - 1], B, uJ, t->widths[L]));
        } else {
            TTRY(forward_layer(t, l, b[l - 1], B, t->Ztmp, t->ldz));
            ctx->launches += 1;
            launch_train_act(s, t->Ztmp, t->ldz, t->widths[l], B, r, t->act, t->X[l & 1]);
        }
    }
    (void)C;
    TCU(ctx, cudaGetLastError());
    return DAE_OK;
}

dae_status dae_train_backward(dae_trainer* t, const float* const* W, const float* const* b, int B,
                              const double* q, const float* g_uJ, double* g_q, float* const* g_W,
                              float* const* g_b) {
    TTRY(check_args(t, W, b, B, q));
    dae_ctx* ctx = t->ctx;
    if (!g_uJ || !on_dev(g_uJ) || !g_W || !g_b)
        return tfail(ctx, DAE_ERR_INVALID_ARG, "cotangents and gradient arrays must be given (device)");
    for (int l = 0; l < t->L; ++l)
        if (!g_W[l] || !g_b[l] || !on_dev(g_W[l]) || !on_dev(g_b[l]))
            return tfail(ctx, DAE_ERR_INVALID_ARG, "gradient arrays must be device arrays");
    if (g_q && !on_dev(g_q)) return tfail(ctx, DAE_ERR_INVALID_ARG, "g_q must be a device array");
    cudaStream_t s = ctx->stream;
    const int L = t->L, r = t->r, C = B * (1 + r);
    const int* w = t->widths.data();
    TTRY(set_batch(t, B));
    stage_weights(t, W, true);
    // forward to the last hidden boundary, keeping the even pre-activations
    ctx->launches += 1;
    launch_train_seed(s, q, B, r, t->X[0]);
    for (int l = 1; l < L; ++l) {
        float* zo = (l % 2 == 0) ? t->Zck[l] : t->Ztmp;
        TTRY(forward_layer(t, l, b[l - 1], B, zo, t->ldz));
        ctx->launches += 1;
        launch_train_act(s, zo, t->ldz, w[l], B, r, t->act, t->X[l & 1]);
    }
    // cotangent of the output layer in both operand layouts
    ctx->launches += 1;
    launch_train_split(s, g_uJ, w[L], B, r, t->Zb);
    const float* zv = g_uJ;          // value rows of the current cotangent
    int zv_ld = w[L];
    for (int l = L; l >= 1; --l) {
        const auto& y = t->layers[l - 1];
        const int k = l - 1;         // boundary feeding layer l
        // X_k in both layouts (recomputed from the nearest checkpoint) and its Z_k
        const float* Zk = nullptr;
        if (l < L) {
            // X_k was produced on the way down; boundary L-1 is current after the forward
            if (k == 0) {
                ctx->launches += 1;
                launch_train_seed(s, q, B, r, t->X[0]);
            } else if (k % 2 == 0) {
                Zk = t->Zck[k];
                ctx->launches += 1;
                launch_train_act(s, Zk, t->ldz, w[k], B, r, t->act, t->X[k & 1]);
            } else {
                // recompute the odd boundary from the even one below it
                if (k - 1 == 0) {
                    ctx->launches += 1;
                    launch_train_seed(s, q, B, r, t->X[0]);
                } else {
                    ctx->launches += 1;
                    launch_train_act(s, t->Zck[k - 1], t->ldz, w[k - 1], B, r, t->act, t->X[(k - 1) & 1]);
                }
                TTRY(forward_layer(t, k, b[k - 1], B, t->Ztmp, t->ldz));
                Zk = t->Ztmp;
                ctx->launches += 1;
                launch_train_act(s, Zk, t->ldz, w[k], B, r, t->act, t->X[k & 1]);
            }
        } else {
            Zk = (k == 0) ? nullptr : ((k % 2 == 0) ? t->Zck[k] : t->Ztmp);
        }
        // W̄_l = Z̄_l X_k^T (contraction over the C batch columns), b̄_l = sum of Z̄_l values
        TTRY(run_gemm(t, gemm(t->tmZn, t->Zb.nf, t->Zb.ldn, t->tmXn[k & 1], t->X[k & 1].nf,
                              t->X[k & 1].ldn, g_W[l - 1], w[k], 0, w[l], w[k],
                              (int)((C + 63) / 64), nullptr, 0, ctx->d_status)));
        ctx->launches += 1;
        launch_train_bias_grad(s, zv, zv_ld, w[l], B, g_b[l - 1]);
        if (l > 1) {
            // X̄_k = W_l^T Z̄_l, then Z̄_k through the activation of boundary k
            TTRY(run_gemm(t, gemm(y.tmWT, y.wtf, y.ldT, t->tmZc, t->Zb.cf, t->Zb.ldc, t->Xbar, t->ldz,
                                  1, w[k], C, y.ldT / 64, nullptr, 0, ctx->d_status)));
            ctx->launches += 1;
            launch_train_act_bwd(s, t->Xbar, t->ldz, Zk, t->ldz, w[k], B, r, t->act, t->Zb, t->zval);
            zv = t->zval;
            zv_ld = w[k];
        } else if (g_q) {
            ctx->launches += 1;
            launch_train_grad_q(s, zv, w[1], W[0], r, B, r, g_q);
        }
    }
    TCU(ctx, cudaGetLastError());
    return DAE_OK;
}

}  // extern "C"
