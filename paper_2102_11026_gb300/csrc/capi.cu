// Host side of the C ABI in include/dae.h: contexts, uploads, argument staging
// and the enqueueing of one evaluation of the reduced system.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <cmath>
#include <vector>

#include <atomic>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <cublas_v2.h>

#include "dae_internal.h"

using namespace dae;

static std::atomic<unsigned long long> g_mesh_ids{1};
static std::atomic<unsigned long long> g_dec_ids{1};

#define DAE_VERSION 10100

namespace {

dae_status fail(dae_ctx* ctx, dae_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

#define CU(ctx, call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DAE_ERR_OOM : DAE_ERR_CUDA,  \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define TRY(x)                          \
    do {                                \
        dae_status s_ = (x);            \
        if (s_ != DAE_OK) return s_;    \
    } while (0)

inline size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

bool on_device(const void* p) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
dae_status dmalloc(dae_ctx* ctx, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) return DAE_OK;
    CU(ctx, cudaMalloc((void**)p, n * sizeof(T)));
    CU(ctx, cudaMemsetAsync(*p, 0, n * sizeof(T), ctx->stream));
    return DAE_OK;
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Per-call staging of host arguments into the context's device arena.
struct Stage {
    dae_ctx* ctx;
    std::vector<char*> host_out;
    std::vector<const char*> dev_out;
    std::vector<size_t> out_bytes;
    size_t used = 0;
    bool any_host = false;
    explicit Stage(dae_ctx* c) : ctx(c) {}

    dae_status reserve(size_t bytes) {
        if (ctx->dstage_bytes >= bytes) return DAE_OK;
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx->dstage);
        size_t nb = std::max(bytes, (size_t)1 << 20);
        CU(ctx, cudaMalloc(&ctx->dstage, nb));
        ctx->dstage_bytes = nb;
        return DAE_OK;
    }
    // Plan: call need() for every host argument first, then reserve(), then map().
    size_t plan = 0;
    void need(const void* p, size_t bytes) {
        if (p && !on_device(p)) plan += round_up(bytes, 256);
    }
    template <class T>
    dae_status in(const T* p, size_t n, const T** out) {
        *out = p;
        if (!p || on_device(p)) return DAE_OK;
        any_host = true;
        char* d = (char*)ctx->dstage + used;
        used += round_up(n * sizeof(T), 256);
        CU(ctx, cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
        *out = (const T*)d;
        return DAE_OK;
    }
    template <class T>
    dae_status inout(T* p, size_t n, T** out, bool copy_in) {
        *out = p;
        if (!p || on_device(p)) return DAE_OK;
        any_host = true;
        char* d = (char*)ctx->dstage + used;
        used += round_up(n * sizeof(T), 256);
        if (copy_in)
            CU(ctx, cudaMemcpyAsync(d, p, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
        host_out.push_back((char*)p);
        dev_out.push_back(d);
        out_bytes.push_back(n * sizeof(T));
        *out = (T*)d;
        return DAE_OK;
    }
    dae_status finish() {
        for (size_t i = 0; i < host_out.size(); ++i)
            CU(ctx, cudaMemcpyAsync(host_out[i], dev_out[i], out_bytes[i], cudaMemcpyDeviceToHost,
                                    ctx->stream));
        if (any_host) CU(ctx, cudaStreamSynchronize(ctx->stream));
        return DAE_OK;
    }
};

dae_status check_device_status(dae_ctx* ctx) {
    int st = 0;
    CU(ctx, cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (st != 0) {
        CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
        // a bounded wait that gave up can leave grid-barrier and split counters mid-count
        if (st == DAE_ERR_TIMEOUT) ctx->timeout_epoch += 1;
        return fail(ctx, (dae_status)st, "device reported %s", dae_status_string((dae_status)st));
    }
    return DAE_OK;
}

// Records a CUDA event pair around one phase when profiling is on.
struct Phase {
    dae_ctx* c;
    int ph;
    cudaEvent_t a = nullptr;
    static cudaEvent_t get(dae_ctx* c) {
        if (!c->ev_pool.empty()) {
            cudaEvent_t e = c->ev_pool.back();
            c->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    Phase(dae_ctx* ctx, int phase, int n_kernels) : c(ctx), ph(phase) {
        c->launches += n_kernels;
        if (c->prof_on & (1u << phase)) {
            a = get(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~Phase() {
        if (a) {
            cudaEvent_t b = get(c);
            cudaEventRecord(b, c->stream);
            c->recs.push_back({ph, a, b});
        }
    }
};

int out_bf16_of(dae_prec p) { return p == DAE_BF16 ? 1 : (p == DAE_BF16X3 ? 2 : 0); }

// ----------------------------------------------------------- workspace --
dae_status alloc_workspace(dae_decoder* d) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    const int r = d->r, L = d->L, N = d->N;
    w.C = n_cols(r);
    w.Cp = pad_cols(r);
    const int sm = ctx->sm_count;
    size_t ldmax = 0, wmax = 0;
    for (int l = 0; l <= L - 1; ++l) ldmax = std::max(ldmax, round_up(d->widths[l], kKPad));
    for (int l = 1; l < L; ++l) wmax = std::max(wmax, (size_t)d->widths[l]);
    w.ldx_max = ldmax;
    for (int i = 0; i < 2; ++i) {
        TRY(dmalloc(ctx, &w.X[i], w.Cp * ldmax));
        TRY(dmalloc(ctx, &w.Xh[i], w.Cp * ldmax));
        TRY(dmalloc(ctx, &w.Xl[i], w.Cp * ldmax));
    }
    w.S1.assign(L - 1, nullptr);
    w.T.assign(L - 1, nullptr);
    for (int l = 0; l < L - 1; ++l) {
        TRY(dmalloc(ctx, &w.S1[l], (size_t)d->widths[l + 1]));
        TRY(dmalloc(ctx, &w.T[l], (size_t)r * d->widths[l + 1]));
    }
    TRY(dmalloc(ctx, &w.u, (size_t)N));
    TRY(dmalloc(ctx, &w.HDD, (size_t)N));
    TRY(dmalloc(ctx, &w.a, (size_t)N));
    TRY(dmalloc(ctx, &w.J, (size_t)r * N));
    TRY(dmalloc(ctx, &w.dJ, (size_t)r * N));
    w.n_row_blocks = (N + 127) / 128;
    w.row_stride = r + r * (r + 1) / 2 + r * r;
    TRY(dmalloc(ctx, &w.row_part, (size_t)w.n_row_blocks * w.row_stride));
    w.row_part_cap = w.n_row_blocks;
    // reverse-pass partials: the largest of the W_L^T a splits and the hidden splits
    const int K = d->widths[L - 1];
    size_t need = (size_t)(128 + kMaxPairSplits + 1) * K;   // dense + pair + f_ext splits
    for (int l = L - 2; l >= 0; --l) {
        int n_o = d->widths[l + 1], n_i = d->widths[l];
        need = std::max(need, (size_t)bwd_split(n_i, n_o, sm) * (1 + r) * n_i);
    }
    w.bwd_part_elems = need;
    TRY(dmalloc(ctx, &w.bwd_part[0], need));
    TRY(dmalloc(ctx, &w.bwd_part[1], need));
    TRY(dmalloc(ctx, &w.gbuf, (size_t)(1 + r) * std::max(wmax, (size_t)1)));
    w.Cb = (int)round_up(1 + r, 16);
    for (int l = 0; l < L - 1; ++l) w.ldg_max = std::max(w.ldg_max, round_up(d->widths[l + 1], kKPad));
    for (int i = 0; i < 2; ++i) {
        TRY(dmalloc(ctx, &w.G32[i], (size_t)w.Cb * w.ldg_max));
        TRY(dmalloc(ctx, &w.Gh[i], (size_t)w.Cb * w.ldg_max));
        TRY(dmalloc(ctx, &w.Gl[i], (size_t)w.Cb * w.ldg_max));
    }
    {
        // split-K scratch of the tensor-core GEMMs: hidden forward layers and the reverse
        // GEMMs (largest tiles x split x columns x 128)
        size_t part = 0, tiles_max = 0;
        for (int l = 0; l < L - 1; ++l) {
            const int m_pad = (int)round_up(d->widths[l + 1], kRowTile);
            const int ldl = (int)round_up(d->widths[l], kKPad);
            const int sp = std::max(tc_split(m_pad, ldl, DAE_BF16, sm), tc_split(m_pad, ldl, DAE_TF32, sm));
            part = std::max(part, (size_t)(m_pad / 128) * sp * w.Cp * 128);
            tiles_max = std::max(tiles_max, (size_t)(m_pad / 128));
            const int mt = (int)round_up(d->widths[l], kRowTile);
            const int ldt = (int)round_up(d->widths[l + 1], kKPad);
            const int spt = std::max(tc_split(mt, ldt, DAE_BF16, sm), tc_split(mt, ldt, DAE_TF32, sm));
            part = std::max(part, (size_t)(mt / 128) * spt * w.Cb * 128);
            tiles_max = std::max(tiles_max, (size_t)(mt / 128));
        }
        TRY(dmalloc(ctx, &w.split_part, std::max(part, (size_t)1)));
        TRY(dmalloc(ctx, &w.split_cnt, std::max(tiles_max, (size_t)1)));
    }
    TRY(dmalloc(ctx, &w.red, red_size(r)));
    TRY(dmalloc(ctx, &w.ns, 1));
    TRY(dmalloc(ctx, &w.lu, (size_t)(kMaxR * kMaxR + 3 * kMaxR)));
    TRY(dmalloc(ctx, &w.qbar, (size_t)r));
    TRY(dmalloc(ctx, &w.qbar_dot, (size_t)r));
    TRY(dmalloc(ctx, &w.q0, (size_t)r));
    TRY(dmalloc(ctx, &w.zvec, (size_t)r));
    TRY(dmalloc(ctx, &w.eval_flag, 1));
    TRY(dmalloc(ctx, &w.f_ext, (size_t)N));
    return DAE_OK;
}

void free_workspace(Workspace& w) {
    for (int i = 0; i < 2; ++i) { dfree(w.X[i]); dfree(w.Xh[i]); dfree(w.Xl[i]); dfree(w.bwd_part[i]); }
    for (int i = 0; i < 2; ++i) { dfree(w.G32[i]); dfree(w.Gh[i]); dfree(w.Gl[i]); }
    for (auto& p : w.S1) dfree(p);
    for (auto& p : w.T) dfree(p);
    dfree(w.u); dfree(w.HDD); dfree(w.a); dfree(w.J); dfree(w.dJ); dfree(w.row_part); dfree(w.out_part);
    dfree(w.Xe[0]); dfree(w.Xe[1]);
    dfree(w.fwd_jobs); dfree(w.rev_jobs); dfree(w.out_job); dfree(w.gbar); dfree(w.chain_part); dfree(w.chain_cnt);
    dfree(w.gbuf); dfree(w.split_part); dfree(w.split_cnt); dfree(w.red); dfree(w.ns); dfree(w.lu); dfree(w.qbar); dfree(w.qbar_dot); dfree(w.q0);
    dfree(w.zvec); dfree(w.eval_flag); dfree(w.f_ext); dfree(w.fe_w); dfree(w.fe_dof);
    dfree(w.cub_part); dfree(w.cub_energy); dfree(w.cub_tets); dfree(w.cub_w); dfree(w.hist);
    if (w.gexec) cudaGraphExecDestroy(w.gexec);
    dfree(w.traj); dfree(w.qout); dfree(w.rc);
    dfree(w.G); dfree(w.xy); dfree(w.pext); dfree(w.fext_prev); dfree(w.pext_flag); dfree(w.pext_part);
    dfree(w.Gs32); dfree(w.Gsh); dfree(w.Gsl); dfree(w.cub_rows); dfree(w.gy); dfree(w.Jc);
    dfree(w.wn_B1); dfree(w.wn_c1); dfree(w.wn_A2); dfree(w.wn_b2); dfree(w.wn_A3); dfree(w.wn_b3);
    dfree(w.wn_A4); dfree(w.wn_b4); dfree(w.wn_h1); dfree(w.wn_w);
    dfree(w.V); dfree(w.UMU); dfree(w.Uf); dfree(w.zpv); dfree(w.lin_part);
}

dae_status ensure_cubature(dae_decoder* d, int n_cub, int n_w) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    const int r = d->np + d->r;   // system size
    w.cub_stride = r + r * (r + 1) / 2;
    if (n_cub > w.cub_cap) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.fe_w); dfree(w.fe_dof); dfree(w.cub_part); dfree(w.cub_energy); dfree(w.cub_tets);
        int cap = std::max(n_cub, 64);
        TRY(dmalloc(ctx, &w.fe_w, (size_t)cap * 12));
        TRY(dmalloc(ctx, &w.fe_dof, (size_t)cap * 12));
        TRY(dmalloc(ctx, &w.cub_part, (size_t)cap * w.cub_stride));
        TRY(dmalloc(ctx, &w.cub_energy, (size_t)cap));
        TRY(dmalloc(ctx, &w.cub_tets, (size_t)cap));
        w.cub_cap = cap;
    }
    if (n_w > w.cub_w_cap) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.cub_w);
        TRY(dmalloc(ctx, &w.cub_w, (size_t)n_w));
        w.cub_w_cap = n_w;
    }
    return DAE_OK;
}

// ----------------------------------------------------------- evaluation --
struct Outs {
    float *u = nullptr, *J = nullptr, *dJ = nullptr, *HDD = nullptr, *Hqq = nullptr;
    // fused row reductions of the output layer (tensor-core path)
    float* row_part = nullptr; int row_stride = 0;
    const float* mdof = nullptr; const float* f_ext = nullptr; float* a_out = nullptr;
    // Gram form (Newton path): the output stage runs over the stacked operand
    bool gram = false; int n_map = 0; const float* pext = nullptr;
};

// Forward-pass arguments of layer l that do not change between calls.
void fill_fwd_args(const dae_decoder* d, int l, FwdArgs& a) {
    const Workspace& w = d->ws;
    const Layer& ly = d->layers[l];
    const int L = d->L;
    memset(&a, 0, sizeof a);
    a.W = ly.W; a.ld = ly.ld; a.Wh = ly.Wh; a.Wl = ly.Wl; a.bias = ly.b;
    a.X = w.X[l & 1]; a.Xh = w.Xh[l & 1]; a.Xl = w.Xl[l & 1];
    a.n_in = ly.n_in; a.n_out = ly.n_out; a.m_pad = ly.m_pad; a.r = d->r; a.Cp = w.Cp;
    a.act = d->act;
    a.last = (l == L - 1);
    a.mode = a.last ? 1 : 0;
    // FP32 activations feed the FP32/TF32 GEMMs and (for the output layer's input) x_y
    // (rounded to TF32 when they feed the tf32 GEMMs)
    a.out_f32 = d->prec == DAE_TF32 ? 2 : ((d->prec == DAE_FP32 || l == L - 2) ? 1 : 0);
    a.tmaps = ly.tm_ok ? (const void*)ly.tm : nullptr;
    a.split_part = w.split_part;
    a.split_cnt = w.split_cnt;
    if (!a.last) {
        a.Y = w.X[(l + 1) & 1]; a.Yh = w.Xh[(l + 1) & 1]; a.Yl = w.Xl[(l + 1) & 1];
        a.ldy = (int)round_up(ly.n_out, kKPad);
        a.out_bf16 = out_bf16_of(d->prec);
        a.S1 = w.S1[l]; a.T = w.T[l];
    }
}

// Reverse-pass arguments of hidden layer l (tensor-core path).
void fill_rev_args(const dae_decoder* d, int l, FwdArgs& a) {
    const Workspace& w = d->ws;
    const Layer& ly = d->layers[l];
    const int L = d->L;
    memset(&a, 0, sizeof a);
    a.ld = ly.ldT; a.m_pad = ly.mT_pad; a.n_in = ly.n_out; a.n_out = ly.n_in;
    a.r = d->r; a.Cp = w.Cb;
    a.tmaps = ly.tmR; a.split_part = w.split_part; a.split_cnt = w.split_cnt;
    if (l > 0) {
        const int nb = (L - 1 - l) & 1;
        a.mode = 2;
        a.Y = w.G32[nb]; a.Yh = w.Gh[nb]; a.Yl = w.Gl[nb];
        a.ldy = d->layers[l - 1].ldT;
        a.out_f32 = (d->prec == DAE_TF32) ? 2 : 0;
        a.out_bf16 = out_bf16_of(d->prec);
        a.S1 = w.S1[l - 1]; a.T = w.T[l - 1];
    } else {
        a.mode = 3;
        a.dout = w.bwd_part[1];
    }
}

// Chain job of hidden forward layer l (whole K loop per 128-row tile).
void make_fwd_job(const dae_decoder* d, int l, ChainJob& j) {
    const Layer& ly = d->layers[l];
    memset(&j, 0, sizeof j);
    memcpy(j.tm, ly.tm, sizeof j.tm);
    fill_fwd_args(d, l, j.a);
    j.tiles = ly.m_pad / 128;
    j.nk = ly.ld / (d->prec == DAE_TF32 ? 32 : 64);
    j.split = 1;
    j.rep = 1;
}

// Chain job of the reverse pass through hidden layer l.
void make_rev_job(const dae_decoder* d, int l, ChainJob& j) {
    const Layer& ly = d->layers[l];
    memset(&j, 0, sizeof j);
    memcpy(j.tm, ly.tmR, sizeof j.tm);
    fill_rev_args(d, l, j.a);
    j.tiles = ly.mT_pad / 128;
    j.nk = ly.ldT / (d->prec == DAE_TF32 ? 32 : 64);
    j.split = 1;
    j.rep = 1;
}

// Chain job of the output layer (outputs and fused row reductions per call).
void make_out_job(const dae_decoder* d, const Outs& o, double dt, double h, ChainJob& job) {
    const Layer& ly = d->layers[d->L - 1];
    memset(&job, 0, sizeof job);
    memcpy(job.tm, ly.tm, sizeof job.tm);
    fill_fwd_args(d, d->L - 1, job.a);
    job.a.inv_h = 1.0 / h; job.a.inv_h2 = 1.0 / (h * h); job.a.inv_h3 = 1.0 / (h * h * h);
    job.a.inv_dt2 = 1.0 / (dt * dt);
    job.a.u = o.u; job.a.J = o.J; job.a.dJ = o.dJ; job.a.HDD = o.HDD; job.a.Hqq = o.Hqq;
    if (o.row_part) {
        job.a.row_part = o.row_part; job.a.row_stride = o.row_stride;
        job.a.mdof = o.mdof; job.a.f_ext = o.f_ext; job.a.zvec = d->ws.zvec; job.a.dt = dt;
        job.a.a_out = o.a_out;
    }
    job.tiles = ly.m_pad / 128;
    job.nk = ly.ld / (d->prec == DAE_TF32 ? 32 : 64);
    job.split = 1;
    job.rep = 1;
    if (o.gram) {
        // [G ; W_L at the cubature DOFs]: reductions over K and the cubature's rows
        const Workspace& w = d->ws;
        memcpy(&job.tm[0], &w.tmGs[0], sizeof(CUtensorMap));
        memcpy(&job.tm[1], &w.tmGs[1], sizeof(CUtensorMap));
        job.tiles = w.Gt + w.Rt;
        job.nk = w.ldGs / (d->prec == DAE_TF32 ? 32 : 64);
        job.a.gram_tiles = w.Gt;
        job.a.K = ly.n_in;
        job.a.row_map = w.cub_rows;
        job.a.n_map = o.n_map;
        job.a.Xg = w.X[(d->L - 1) & 1];
        job.a.ldxg = ly.ld;
        job.a.pext = o.pext;
        job.a.gy = w.gy;
        job.a.a_out = nullptr;
        job.a.Jc = w.Jc;
        job.a.ldc = w.Rt * 128;
    }
}

// Gram form of the Newton path's output stage: available for the tensor-core
// precisions once G is formed for this mesh.
bool gram_out(const dae_decoder* d, const dae_mesh* m) {
    const Workspace& w = d->ws;
    return d->prec != DAE_FP32 && w.chain_ok && w.gs_ok && w.G && w.G_mesh == m->id &&
           w.gs_G_mesh == m->id;
}

// The stacked operand [G ; cubature rows of W_L] (allocation, tensor maps, G part).
dae_status ensure_gs(dae_decoder* d, const dae_mesh* m, int n_cub) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (d->prec == DAE_FP32 || !w.chain_ok || !w.G || w.G_mesh != m->id) return DAE_OK;
    const Layer& top = d->layers[d->L - 1];
    const int K = top.n_in;
    const int Gt = (K + 127) / 128, Rt = (12 * n_cub + 127) / 128;
    const int rows = (Gt + Rt) * 128;
    const bool f32 = d->prec == DAE_TF32, x3 = d->prec == DAE_BF16X3;
    const bool have = f32 ? w.Gs32 != nullptr : (w.Gsh != nullptr && (!x3 || w.Gsl));
    if (!have || rows > w.gs_rows_cap || w.ldGs != top.ld) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.Gs32); dfree(w.Gsh); dfree(w.Gsl); dfree(w.cub_rows);
        const size_t n = (size_t)rows * top.ld;
        if (f32) {
            TRY(dmalloc(ctx, &w.Gs32, n));
            CU(ctx, cudaMemsetAsync(w.Gs32, 0, n * sizeof(float), ctx->stream));
        } else {
            TRY(dmalloc(ctx, &w.Gsh, n));
            CU(ctx, cudaMemsetAsync(w.Gsh, 0, n * sizeof(__nv_bfloat16), ctx->stream));
            if (x3) {
                TRY(dmalloc(ctx, &w.Gsl, n));
                CU(ctx, cudaMemsetAsync(w.Gsl, 0, n * sizeof(__nv_bfloat16), ctx->stream));
            }
        }
        TRY(dmalloc(ctx, &w.cub_rows, (size_t)rows));
        CU(ctx, cudaMemsetAsync(w.cub_rows, 0xff, (size_t)rows * sizeof(int), ctx->stream));
        if (!w.gy) TRY(dmalloc(ctx, &w.gy, (size_t)K));
        w.gs_rows_cap = rows;
        w.ldGs = top.ld;
        w.gs_G_mesh = 0;
        bool ok = make_tmap(&w.tmGs[0], f32 ? (const void*)w.Gs32 : (const void*)w.Gsh, f32, w.ldGs,
                            rows, 128);
        if (x3) ok = ok && make_tmap(&w.tmGs[1], w.Gsl, false, w.ldGs, rows, 128);
        else w.tmGs[1] = w.tmGs[0];
        if (!ok) return fail(ctx, DAE_ERR_UNSUPPORTED, "tensor map encoding failed (Gram operand)");
        w.graph_ok = false;
    }
    // one arrival counter per output tile of the stacked operand; checked on every call,
    // since rebuilding the layer chains (a precision change) resizes the counters to the
    // hidden layers' and the row form's needs only
    if (w.chain_cnt_n < (size_t)(Gt + Rt + 1)) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.chain_cnt);
        w.chain_cnt_n = Gt + Rt + 1;
        TRY(dmalloc(ctx, &w.chain_cnt, w.chain_cnt_n));
        w.graph_ok = false;
    }
    // the cubature rows' u and J in compact form (written by the output stage)
    const size_t jc = (size_t)(1 + d->r) * Rt * 128;
    if (jc > w.Jc_cap) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.Jc);
        TRY(dmalloc(ctx, &w.Jc, jc));
        w.Jc_cap = jc;
        w.graph_ok = false;
    }
    // the stream-form output stage stores its items unfinished (k_out_finish sums and
    // finishes them): raw_m slots per CTA, the most tiles one CTA's k-block range touches
    {
        const int G = ctx->sm_count;
        const long long nk = w.ldGs / (f32 ? 32 : 64);
        const long long T = (long long)(Gt + Rt) * nk;
        int mx = 0;
        if (T >= G)
            for (int c = 0; c < G; ++c) {
                const long long a = T * c / G, b = T * (c + 1) / G;
                mx = std::max(mx, (int)((b - 1) / nk - a / nk + 1));
            }
        const size_t need = (size_t)G * mx * 128 * (w.Cp + 1);
        if (need > w.out_part_cap) {
            CU(ctx, cudaStreamSynchronize(ctx->stream));
            dfree(w.out_part);
            TRY(dmalloc(ctx, &w.out_part, need));
            w.out_part_cap = need;
            w.graph_ok = false;
        }
        w.raw_m = mx;
        const int rows = kFinishBlocks * Gt;   // partial rows of the finish kernel
        if (rows > w.row_part_cap) {
            CU(ctx, cudaStreamSynchronize(ctx->stream));
            dfree(w.row_part);
            TRY(dmalloc(ctx, &w.row_part, (size_t)rows * w.row_stride));
            w.row_part_cap = rows;
            w.graph_ok = false;
        }
    }
    if (w.gs_G_mesh != m->id) {
        const size_t n = (size_t)K * w.ldGs;   // G is [K][ldG], ldG = ldGs
        if (f32) launch_round_tf32(ctx->stream, w.G, w.Gs32, n);
        else launch_split_bf16(ctx->stream, w.G, w.Gsh, x3 ? w.Gsl : nullptr, n);
        CU(ctx, cudaGetLastError());
        w.gs_G_mesh = m->id;
    }
    w.Gt = Gt;
    w.Rt = Rt;
    w.gs_ok = true;
    return DAE_OK;
}

GatherArgs gs_gather_args(const dae_decoder* d, const dae_mesh* m, int n_cub) {
    const Workspace& w = d->ws;
    const Layer& top = d->layers[d->L - 1];
    GatherArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.cub_tets = w.cub_tets; ga.tets = m->tets; ga.n_cub = n_cub; ga.n_rows = w.Rt * 128;
    ga.ld = w.ldGs; ga.row0 = w.Gt * 128; ga.map = w.cub_rows;
    if (d->prec == DAE_TF32) {
        ga.src32 = top.Wr; ga.dst32 = w.Gs32;
    } else {
        ga.srch = top.Wh; ga.dsth = w.Gsh;
        if (d->prec == DAE_BF16X3) { ga.srcl = top.Wl; ga.dstl = w.Gsl; }
    }
    return ga;
}

// Per call, after the cubature tets are staged: the stacked operand's cubature rows.
dae_status prepare_gram_out(dae_decoder* d, const dae_mesh* m, int n_cub) {
    TRY(ensure_gs(d, m, n_cub));
    if (!gram_out(d, m)) return DAE_OK;
    d->ctx->launches += 1;
    launch_gather_cub_rows(d->ctx->stream, nullptr, gs_gather_args(d, m, n_cub), 1);
    CU(d->ctx, cudaGetLastError());
    return DAE_OK;
}

// Plan of chain layer l (direction dir): the decoder's stored plan for its precision,
// else the fixed heuristic.
void apply_plan(const dae_decoder* d, int dir, int l, ChainJob& j, int grid) {
    const auto& sp = d->plan_split[dir];
    j.solo = 0;
    if (d->plan_prec == (int)d->prec && (int)sp.size() == d->L - 1) {
        j.split = sp[l];
        j.rep = d->plan_rep[dir][l];
        if (j.rep == 0) {          // solo: the whole layer on CTA 0
            j.rep = 1;
            j.solo = 1;
        }
    } else {
        chain_plan(j, grid);
    }
}

// The job lists of both directions with the current plans; part = floats of split-K
// partial tiles they need, cnt = their per-tile counters.
void chain_jobs(const dae_decoder* d, std::vector<ChainJob>& fj, std::vector<ChainJob>& rj,
                size_t& part, size_t& cnt_f, size_t& cnt_r) {
    const Workspace& w = d->ws;
    const int L = d->L, G = d->ctx->sm_count;
    fj.assign(L - 1, ChainJob{});
    rj.assign(L - 1, ChainJob{});
    part = 1;
    cnt_f = cnt_r = 0;
    for (int l = 0; l < L - 1; ++l) {
        ChainJob& j = fj[l];
        make_fwd_job(d, l, j);
        apply_plan(d, 0, l, j, G);
        j.cnt_off = (int)cnt_f;
        cnt_f += j.tiles;
        part = std::max(part, (size_t)j.tiles * j.split * (w.Cp + 1) * 128);
    }
    for (int i = 0; i < L - 1; ++i) {
        const int l = L - 2 - i;
        ChainJob& j = rj[i];
        make_rev_job(d, l, j);
        apply_plan(d, 1, l, j, G);
        j.cnt_off = (int)cnt_r;
        cnt_r += j.tiles;
        part = std::max(part, (size_t)j.tiles * j.split * (w.Cb + 1) * 128);
    }
    // the per-tile ready counters follow the split counters in the same array
    cnt_f = (cnt_f + kRdyStride - 1) / kRdyStride * kRdyStride;
    cnt_r = (cnt_r + kRdyStride - 1) / kRdyStride * kRdyStride;
    for (auto& j : fj) { j.rdy_off = (int)cnt_f; cnt_f += (size_t)j.tiles * kRdyStride; }
    for (auto& j : rj) { j.rdy_off = (int)cnt_r; cnt_r += (size_t)j.tiles * kRdyStride; }
}

// Job lists of the persistent layer-chain kernel (both directions).
dae_status build_chains(dae_decoder* d) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    const int L = d->L, G = ctx->sm_count;
    std::vector<ChainJob> fj, rj;
    size_t part, cnt_f, cnt_r;
    chain_jobs(d, fj, rj, part, cnt_f, cnt_r);
    if (!w.fwd_jobs) {
        // the hidden layers, and a slot for the output stage run as the chain's last job
        CU(ctx, cudaMalloc(&w.fwd_jobs, sizeof(ChainJob) * L));
        CU(ctx, cudaMalloc(&w.rev_jobs, sizeof(ChainJob) * (L - 1)));
        CU(ctx, cudaMalloc(&w.out_job, sizeof(ChainJob)));
        TRY(dmalloc(ctx, &w.gbar, 1));
    }
    // the output layer's stream pieces: two partial tiles per CTA, a counter per tile
    const Layer& top = d->layers[L - 1];
    part = std::max(part, (size_t)G * 2 * (w.Cp + 1) * 128);
    dfree(w.chain_part);
    TRY(dmalloc(ctx, &w.chain_part, part));
    dfree(w.chain_cnt);
    w.chain_cnt_n = std::max(std::max(cnt_f, cnt_r), (size_t)(top.m_pad / 128)) + 1;
    TRY(dmalloc(ctx, &w.chain_cnt, w.chain_cnt_n));
    CU(ctx, cudaMemcpy(w.fwd_jobs, fj.data(), sizeof(ChainJob) * (L - 1), cudaMemcpyHostToDevice));
    CU(ctx, cudaMemcpy(w.rev_jobs, rj.data(), sizeof(ChainJob) * (L - 1), cudaMemcpyHostToDevice));
    w.chain_ok = true;
    return DAE_OK;
}

// ------------------------------------------------------------ autotuner --
// Candidate plans of one chain layer: P = 1, 2, 4 or 8 CTAs per 128-row tile (tiles x P
// within the grid), each as replicated K loops or (P >= 2) as a K split with at least
// two k-blocks per chunk; and, for a small layer, every tile on CTA 0 (rep 0: solo).
std::vector<std::pair<int, int>> plan_candidates(const ChainJob& j, int grid) {
    std::vector<std::pair<int, int>> c;   // (split, rep); rep 0: solo
    for (int P = 1; P <= 8; P *= 2) {
        if (j.tiles * P > grid) break;
        c.push_back({1, P});
        if (P >= 2 && j.nk >= 2 * P) c.push_back({P, 1});
    }
    // small layers on CTA 0 alone (the other CTAs skip them)
    if (j.tiles <= 8 && j.tiles * j.nk <= 64) c.push_back({1, 0});
    return c;
}

// Mean device time (ms) of one launch of a direction's chain with the given job list,
// over `reps` back-to-back launches after two warm-up launches (CUDA events on the
// context's stream).  The buffers hold whatever the last evaluation left: the time of a
// chain does not depend on the values.
dae_status time_chain(dae_decoder* d, int dir, const std::vector<ChainJob>& jobs, int reps,
                      double* ms) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    const int L = d->L;
    ChainJob* dst = dir == 0 ? w.fwd_jobs : w.rev_jobs;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    CU(ctx, cudaMemcpy(dst, jobs.data(), sizeof(ChainJob) * (L - 1), cudaMemcpyHostToDevice));
    ChainLaunch cl = {};
    cl.jobs = dst; cl.n_jobs = L - 1; cl.Cp = dir == 0 ? w.Cp : w.Cb; cl.grid = ctx->sm_count;
    cl.gb = w.gbar; cl.ns = nullptr; cl.status = ctx->d_status; cl.split_part = w.chain_part;
    cl.split_cnt = w.chain_cnt;
    cudaEvent_t e0, e1;
    CU(ctx, cudaEventCreate(&e0));
    CU(ctx, cudaEventCreate(&e1));
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) ok = launch_chain(ctx->stream, cl, d->prec);
    cudaEventRecord(e0, ctx->stream);
    for (int i = 0; i < reps && ok; ++i) ok = launch_chain(ctx->stream, cl, d->prec);
    cudaEventRecord(e1, ctx->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->launches += 2 + reps;
    if (!ok) return fail(ctx, DAE_ERR_CUDA, "chain launch failed while tuning");
    if (e != cudaSuccess) return fail(ctx, DAE_ERR_CUDA, "chain timing: %s", cudaGetErrorString(e));
    TRY(check_device_status(ctx));
    *ms = t / reps;
    return DAE_OK;
}

// Validated plan of one direction (sizes L - 1): every layer's (split, rep) must be a
// candidate of plan_candidates.
dae_status check_plan(dae_decoder* d, int dir, const int* split, const int* rep) {
    std::vector<ChainJob> fj, rj;
    size_t part, cf, cr;
    chain_jobs(d, fj, rj, part, cf, cr);
    const std::vector<ChainJob>& jobs = dir == 0 ? fj : rj;
    for (int l = 0; l < d->L - 1; ++l) {
        const ChainJob& j = jobs[dir == 0 ? l : d->L - 2 - l];
        bool found = false;
        for (auto c : plan_candidates(j, d->ctx->sm_count)) found |= (c.first == split[l] && c.second == rep[l]);
        if (!found)
            return fail(d->ctx, DAE_ERR_INVALID_ARG, "layer %d: (split %d, rep %d) is not a valid plan", l,
                        split[l], rep[l]);
    }
    return DAE_OK;
}

dae_status enqueue_forward(dae_decoder* d, const NewtonState* ns, const double* q_override,
                           double dt, double h, int mode, const Outs& o, int off = 0) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    cudaStream_t s = ctx->stream;
    const int r = d->r, L = d->L;
    const int ob = out_bf16_of(d->prec);
    const int ld0 = (int)round_up(r, kKPad);
    {
        Phase p(ctx, DAE_PHASE_SEED, 1);
        launch_seed(s, ns, q_override, w.qbar + off, w.qbar_dot + off, dt, h, mode, r, w.Cp, ld0,
                    w.X[0], w.Xh[0], w.Xl[0], d->prec == DAE_TF32 ? kStoreTF32 : ob, w.zvec, off);
    }
    const bool chain = d->ws.chain_ok;
    if (chain) {
        // the output layer's job: a stream of k-block ranges per CTA when the tiles do not
        // divide evenly over the grid (and the Gram form's few long tiles), provided every
        // CTA gets at least one k-block (a tile's finisher counts one piece from each CTA
        // its k-blocks span)
        ChainJob job;
        make_out_job(d, o, dt, h, job);
        const long long T = (long long)job.tiles * job.nk;
        job.stream = (T >= ctx->sm_count && (job.tiles > ctx->sm_count || o.gram)) ? 1 : 0;
        job.cnt_off = 0;
        // the Gram form's items go out unfinished and a second kernel sums and finishes
        // them with many CTAs: no CTA of the stream waits for another's pieces, and the
        // rows' reductions run on all SMs instead of on one CTA per tile.  That output
        // stage then runs as the last job of the hidden chain's launch: its k-blocks start
        // as soon as the last hidden layer's tiles holding their rows are written
        job.raw = (o.gram && job.stream && w.raw_m > 0) ? 1 : 0;
        job.raw_m = job.raw ? w.raw_m : 0;
        job.raw_part = job.raw ? w.out_part : nullptr;
        const bool fuse = job.raw != 0;
        if (fuse) {
            ctx->launches += 1;
            launch_store_job(s, w.fwd_jobs + (L - 1), job);
        }
        {
            ChainLaunch cl = {};
            cl.jobs = w.fwd_jobs; cl.n_jobs = fuse ? L : L - 1; cl.Cp = w.Cp; cl.grid = ctx->sm_count;
            cl.gb = w.gbar; cl.ns = ns; cl.status = ctx->d_status; cl.split_part = w.chain_part;
            cl.split_cnt = w.chain_cnt;
            Phase p(ctx, DAE_PHASE_FWD_HIDDEN, 1);
            if (!launch_chain(s, cl, d->prec))
                return fail(ctx, DAE_ERR_CUDA, "layer-chain launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
        if (fuse) {
            Phase p(ctx, DAE_PHASE_FWD_OUT, 1);
            launch_out_finish(s, w.fwd_jobs + (L - 1), job.tiles, w.Cp, w.out_part, ctx->sm_count, ns);
        } else {
            ctx->launches += 1;
            launch_store_job(s, w.out_job, job);
            ChainLaunch cl = {};
            cl.jobs = w.out_job; cl.n_jobs = 1; cl.Cp = w.Cp; cl.grid = ctx->sm_count;
            cl.gb = w.gbar; cl.ns = ns; cl.status = ctx->d_status; cl.split_part = w.chain_part;
            cl.split_cnt = w.chain_cnt;
            Phase p(ctx, DAE_PHASE_FWD_OUT, 1);
            if (!launch_chain(s, cl, d->prec))
                return fail(ctx, DAE_ERR_CUDA, "output-layer launch failed: %s", cudaGetErrorString(cudaGetLastError()));
        }
    }
    for (int l = chain ? L : 0; l < L; ++l) {
        FwdArgs a;
        fill_fwd_args(d, l, a);
        a.ns = ns;
        a.status = ctx->d_status;
        a.inv_h = 1.0 / h; a.inv_h2 = 1.0 / (h * h); a.inv_h3 = 1.0 / (h * h * h);
        a.inv_dt2 = 1.0 / (dt * dt);
        if (a.last) {
            a.u = o.u; a.J = o.J; a.dJ = o.dJ; a.HDD = o.HDD; a.Hqq = o.Hqq;
            if (d->prec != DAE_FP32 && o.row_part) {
                a.row_part = o.row_part; a.row_stride = o.row_stride;
                a.mdof = o.mdof; a.f_ext = o.f_ext; a.zvec = w.zvec; a.dt = dt; a.a_out = o.a_out;
            }
        }
        Phase p(ctx, a.last ? DAE_PHASE_FWD_OUT : DAE_PHASE_FWD_HIDDEN, 1);
        if (d->prec == DAE_FP32) {
            launch_fwd_simt(s, a);
        } else if (!launch_fwd_tc(s, a, d->prec, ctx->sm_count)) {
            return fail(ctx, DAE_ERR_UNSUPPORTED, "precision %d not available for layer %d", d->prec, l);
        }
    }
    CU(ctx, cudaGetLastError());
    return DAE_OK;
}

bool use_gram(const dae_decoder* d) {
    const size_t K = d->widths[d->L - 1];
    return 2 * K <= (size_t)d->N;
}

// G = W_L^T diag(m) W_L (set-up, once per decoder/mesh pair; cuBLAS SGEMM in FP32 over row chunks)
dae_status ensure_linear_terms(dae_decoder* d, const dae_mesh* m);

dae_status ensure_gram(dae_decoder* d, const dae_mesh* m) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (w.G && w.G_mesh == m->id) return ensure_linear_terms(d, m);
    const Layer& top = d->layers[d->L - 1];
    const int K = top.n_in, N = top.n_out;
    if (!w.G) {
        w.ldG = (int)round_up(K, kKPad);
        TRY(dmalloc(ctx, &w.G, (size_t)K * w.ldG));
        TRY(dmalloc(ctx, &w.xy, (size_t)w.ldG));
    }
    if (!ctx->cublas) {
        cublasHandle_t hnd;
        if (cublasCreate(&hnd) != CUBLAS_STATUS_SUCCESS) return fail(ctx, DAE_ERR_CUDA, "cublasCreate failed");
        ctx->cublas = hnd;
    }
    cublasHandle_t hnd = (cublasHandle_t)ctx->cublas;
    cublasSetStream(hnd, ctx->stream);
    cublasSetMathMode(hnd, CUBLAS_DEFAULT_MATH);
    const int CH = 4096;
    float* tmp = nullptr;
    TRY(dmalloc(ctx, &tmp, (size_t)CH * top.ld));
    for (int n0 = 0; n0 < N; n0 += CH) {
        const int rows = std::min(CH, N - n0);
        launch_scale_rows(ctx->stream, top.W + (size_t)n0 * top.ld, top.ld, m->mdof + n0, rows, tmp);
        const float one = 1.f, beta = n0 == 0 ? 0.f : 1.f;
        // column-major view: Wc = W^T (K x rows, ld), G += Wc (Wc diag(m))^T
        cublasStatus_t st = cublasSgemm(hnd, CUBLAS_OP_N, CUBLAS_OP_T, K, K, rows, &one,
                                        top.W + (size_t)n0 * top.ld, top.ld, tmp, top.ld, &beta,
                                        w.G, w.ldG);
        if (st != CUBLAS_STATUS_SUCCESS) {
            cudaFree(tmp);
            return fail(ctx, DAE_ERR_CUDA, "cublasSgemm failed (%d)", (int)st);
        }
    }
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(tmp);
    w.G_mesh = m->id;
    return ensure_linear_terms(d, m);
}

// Linear subspace, per mesh: V = W_L^T M U ([ld][np]) and U^T M U ([np][np]), FP32 cuBLAS.
dae_status ensure_linear_terms(dae_decoder* d, const dae_mesh* m) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (d->np == 0 || w.V_mesh == m->id) return DAE_OK;
    const Layer& top = d->layers[d->L - 1];
    const int N = d->N, np = d->np;
    cublasHandle_t hnd = (cublasHandle_t)ctx->cublas;
    cublasSetStream(hnd, ctx->stream);
    cublasSetMathMode(hnd, CUBLAS_DEFAULT_MATH);
    float* MU = nullptr;
    TRY(dmalloc(ctx, &MU, (size_t)np * N));
    // MU[a][n] = m_n U[a][n]: U rows are the first np rows of J ([np][N] = column-major N x np)
    for (int a = 0; a < np; ++a)
        launch_scale_rows(ctx->stream, w.J + (size_t)a * N, 1, m->mdof, N, MU + (size_t)a * N);
    const float one = 1.f, zero = 0.f;
    // V (column-major np x ld, = row-major [ld][np]) = (MU)^T W_L,  U^T M U = (MU)^T U
    cublasStatus_t cs = cublasSgemm(hnd, CUBLAS_OP_T, CUBLAS_OP_T, np, top.ld, N, &one, MU, N, top.W,
                                    top.ld, &zero, w.V, np);
    if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasSgemm(hnd, CUBLAS_OP_T, CUBLAS_OP_N, np, np, N, &one, MU, N, w.J, N, &zero, w.UMU, np);
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(MU);
    if (cs != CUBLAS_STATUS_SUCCESS) return fail(ctx, DAE_ERR_CUDA, "linear-subspace set-up failed (%d)", (int)cs);
    w.V_mesh = m->id;
    return DAE_OK;
}

dae_status ensure_pext_bufs(dae_decoder* d) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (w.pext) return DAE_OK;
    const Layer& top = d->layers[d->L - 1];
    const int K = top.n_in, N = top.n_out;
    const int kb = (K + 1023) / 1024;
    const int splits = std::max(1, std::min(128, std::min((N + 63) / 64, (4 * ctx->sm_count + kb - 1) / kb)));
    TRY(dmalloc(ctx, &w.pext, (size_t)K + 4));
    TRY(dmalloc(ctx, &w.fext_prev, (size_t)N));
    TRY(dmalloc(ctx, &w.pext_flag, 1));
    TRY(dmalloc(ctx, &w.pext_part, (size_t)splits * K));
    w.pext_splits = splits;
    return DAE_OK;
}

// W_L^T f_ext, recomputed on the device only when f_ext differs from the cached copy.
dae_status prepare_pext(dae_decoder* d, const float* f_ext_dev) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (!f_ext_dev) return DAE_OK;
    const Layer& top = d->layers[d->L - 1];
    const int K = top.n_in, N = top.n_out;
    TRY(ensure_pext_bufs(d));
    if (!w.pext_valid) {
        const int one = 1;
        CU(ctx, cudaMemcpyAsync(w.pext_flag, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (d->np > 0) {
        // U^T f_ext for the linear subspace's rows of phi
        const float one = 1.f, zero = 0.f;
        cublasHandle_t hnd = (cublasHandle_t)ctx->cublas;
        cublasSetStream(hnd, ctx->stream);
        if (cublasSgemv(hnd, CUBLAS_OP_T, N, d->np, &one, w.J, N, f_ext_dev, 1, &zero, w.Uf, 1) !=
            CUBLAS_STATUS_SUCCESS)
            return fail(ctx, DAE_ERR_CUDA, "U^T f_ext failed");
    }
    ctx->launches += 4;
    launch_fext_check(ctx->stream, f_ext_dev, w.fext_prev, N, w.pext_flag);
    WtaArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.W = top.W; wa.ld = top.ld; wa.N = N; wa.K = K; wa.a = f_ext_dev;
    wa.nsplit_dense = w.pext_splits; wa.nsplit_pairs = 0; wa.run_flag = w.pext_flag;
    wa.part = w.pext_part;
    launch_wta(ctx->stream, wa);
    launch_pext_finish(ctx->stream, w.pext_part, w.pext_splits, K, w.pext, f_ext_dev, w.fext_prev, N,
                       w.pext_flag);
    CU(ctx, cudaGetLastError());
    w.pext_valid = true;
    return DAE_OK;
}

struct EvalParams {
    double dt, h;
    const int* cub_tets; const float* cub_w; int n_cub;
    int w_stride;             // cubature weights per frame
    const float* f_ext;       // device, may be null
    int control;
    const dae_newton_opts* opts;
    cudaGraphConditionalHandle hcond = 0;
    int use_cond = 0;
    unsigned long long* kcount = nullptr;
    int kpe = 0;
    int wnet = 0;             // predict the cubature weights (first evaluation of a frame)
};

WnetArgs wnet_args(const dae_decoder* d, const int* tets, int n, float* w_out,
                   const NewtonState* ns, int first_only) {
    const Workspace& w = d->ws;
    const Layer& top = d->layers[d->L - 1];
    WnetArgs a;
    memset(&a, 0, sizeof a);
    a.x = w.X[(d->L - 1) & 1]; a.K = top.n_in; a.ldx = top.ld;
    a.B1 = w.wn_B1; a.c1 = w.wn_c1; a.H1 = w.wn_H1;
    a.A2 = w.wn_A2; a.b2 = w.wn_b2; a.H2 = w.wn_H2;
    a.A3 = w.wn_A3; a.b3 = w.wn_b3; a.H3 = w.wn_H3;
    a.A4 = w.wn_A4; a.b4 = w.wn_b4;
    a.tets = tets; a.n = n; a.h1 = w.wn_h1; a.w = w_out;
    a.ns = ns; a.first_only = first_only;
    return a;
}

dae_status enqueue_eval(dae_decoder* d, const dae_mesh* m, NewtonState* ns,
                        const double* q_override, const EvalParams& P) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    cudaStream_t s = ctx->stream;
    const int r = d->r, L = d->L, N = d->N;
    const int np = d->np, n = np + r;   // linear basis size, system size
    const int sm = ctx->sm_count;
    Outs o;
    // the decoder's J follows the np rows of the linear basis U in the J buffer
    o.u = w.u; o.J = w.J + (size_t)np * N; o.dJ = w.dJ; o.HDD = w.HDD;
    const bool fused_rows = d->prec != DAE_FP32;
    const bool gout = gram_out(d, m);
    if (fused_rows) {
        o.row_part = w.row_part; o.row_stride = w.row_stride;
        o.mdof = m->mdof; o.f_ext = P.f_ext; o.a_out = w.a;
    }
    if (gout) {
        o.gram = true;
        o.n_map = 12 * P.n_cub;
        o.pext = P.f_ext ? w.pext : nullptr;
    }
    TRY(enqueue_forward(d, ns, q_override, P.dt, P.h, SEED_FULL, o, np));
    if (P.wnet && P.n_cub > 0) {
        // cubature weights of this frame from the weight network at its first iterate
        Phase p(ctx, DAE_PHASE_CUBATURE, 3);
        launch_wnet(s, wnet_args(d, P.cub_tets, P.n_cub, const_cast<float*>(P.cub_w), ns,
                                 P.control ? 1 : 0));
    }
    if (!fused_rows) {
    RowArgs ra;
    ra.J = w.J; ra.dJ = w.dJ; ra.HDD = w.HDD; ra.mdof = m->mdof; ra.f_ext = P.f_ext;
    ra.zvec = w.zvec; ra.a = w.a; ra.part = w.row_part; ra.N = N; ra.r = r;
    ra.stride = w.row_stride; ra.dt = P.dt; ra.ns = ns;
    {
        Phase p(ctx, DAE_PHASE_ROWS, 1);
        launch_row_reduce(s, ra, w.n_row_blocks);
    }
    }
    // wta arguments first: the linear-subspace kernel writes one of its seed rows
    const Layer& top = d->layers[L - 1];
    const int K = top.n_in;
    const int kb = (K + 1023) / 1024;
    const bool gram = w.G && w.G_mesh == m->id;
    WtaArgs wa;
    memset(&wa, 0, sizeof wa);
    wa.fe_w = w.fe_w; wa.fe_dof = w.fe_dof; wa.n_pairs = 12 * P.n_cub; wa.dt2 = P.dt * P.dt;
    wa.Wp = top.W; wa.ldp = top.ld; wa.K = K;
    if (gram) {
        wa.W = w.G; wa.ld = w.ldG; wa.N = K; wa.a = w.xy;
        wa.pext = P.f_ext ? w.pext : nullptr;
        wa.pext_scale = (float)(-P.dt * P.dt);
    } else {
        wa.W = top.W; wa.ld = top.ld; wa.N = N; wa.a = w.a;
    }
    wa.nsplit_dense = std::max(1, std::min(128, std::min((wa.N + 63) / 64, (4 * sm + kb - 1) / kb)));
    wa.nsplit_pairs = std::max(1, std::min(kMaxPairSplits, (wa.n_pairs + 15) / 16));
    wa.part = w.bwd_part[0]; wa.ns = ns;
    if (gout) {
        // W_L^T M y = G x_y came out of the output stage
        wa.W = nullptr; wa.nsplit_dense = 0; wa.gy = w.gy;
    }
    int in_split = wa.nsplit_dense + wa.nsplit_pairs + (wa.pext ? 1 : 0) + (wa.gy ? 1 : 0);
    if (np > 0) {
        // V^T X partials (U^T M J, U^T M dJ, U^T M y) and the seed row W_L^T M U z_p
        LinArgs la;
        la.X = w.X[(L - 1) & 1]; la.K = K; la.ldx = top.ld; la.r = r; la.np = np;
        la.V = w.V; la.part = w.lin_part; la.vz = w.bwd_part[0] + (size_t)in_split * K;
        la.zpv = w.zpv; la.ns = ns; la.q_in = q_override; la.qbar = w.qbar;
        la.qbar_dot = w.qbar_dot; la.dt = P.dt;
        Phase p(ctx, DAE_PHASE_CUBATURE, 1);
        launch_linear(s, la, w.lin_blocks);
        in_split += 1;
    }
    CubArgs ca;
    ca.w_stride = P.w_stride;
    ca.np = np; ca.pv = np > 0 ? w.zpv + np : nullptr;
    ca.u = w.u; ca.J = w.J; ca.N = N; ca.r = n; ca.X = m->X; ca.tets = m->tets; ca.Bm = m->Bm;
    ca.vol = m->vol; ca.n_tet = m->n_tet; ca.material = m->material; ca.mu = (float)m->mu; ca.lam = (float)m->lam;
    ca.cub_tets = P.cub_tets; ca.cub_w = P.cub_w; ca.n_cub = P.n_cub;
    ca.fe_w = w.fe_w; ca.fe_dof = w.fe_dof; ca.part = w.cub_part; ca.energy = w.cub_energy;
    ca.stride = w.cub_stride; ca.ns = ns; ca.eval_flag = w.eval_flag;
    ca.Jc = gout ? w.Jc : nullptr; ca.ldc = w.Rt * 128;
    ca.n_parts = cubature_parts(P.n_cub, sm);
    {
        Phase p(ctx, DAE_PHASE_CUBATURE, P.n_cub > 0 ? 1 : 0);
        launch_cubature(s, ca);
    }
    if (L == 1)
        return fail(ctx, DAE_ERR_UNSUPPORTED, "a decoder needs at least one hidden layer");
    // phi, the energy and the line-search decision: under Newton control, an iterate that
    // is not accepted for a new Newton step skips the reverse pass and A below
    AsmArgs aa;
    memset(&aa, 0, sizeof aa);
    aa.r = n; aa.dt = P.dt; aa.h = P.h;
    aa.rq = r; aa.np = np; aa.lin_part = w.lin_part; aa.lin_blocks = w.lin_blocks;
    aa.UMU = w.UMU; aa.Uf = P.f_ext ? w.Uf : nullptr; aa.qbar = w.qbar; aa.qbar_dot = w.qbar_dot;
    aa.q_in = q_override;
    aa.row_part = w.row_part;
    aa.n_row_blocks = gout ? (w.raw_m > 0 ? kFinishBlocks * w.Gt : w.Gt) : w.n_row_blocks;
    aa.row_stride = w.row_stride;
    aa.cub_part = w.cub_part; aa.cub_energy = w.cub_energy; aa.n_cub = P.n_cub;
    aa.cub_stride = w.cub_stride; aa.cub_parts = ca.n_parts;
    aa.red = w.red; aa.ns = ns; aa.control = P.control;
    if (P.opts) {
        aa.tol = P.opts->tol; aa.c_armijo = P.opts->c_armijo; aa.max_iter = P.opts->max_iter;
        aa.max_step = P.opts->max_step; aa.xtol = P.opts->xtol;
        aa.max_halvings = P.opts->max_halvings; aa.max_evals = P.opts->max_evals;
    }
    aa.eval_flag = w.eval_flag; aa.status = ctx->d_status;
    aa.lu = P.control ? w.lu : nullptr;
    aa.hcond = P.hcond; aa.use_cond = P.use_cond; aa.kcount = P.kcount; aa.kpe = P.kpe;
    {
        Phase p(ctx, DAE_PHASE_ASSEMBLE, 2);
        launch_decide(s, aa);
    }
    // delta_{L-1} = W_L^T a = W_L^T M y - dt^2 W_L^T f_ext + dt^2 W_L^T f_C:
    // with the Gram matrix, W_L^T M y = G x_y (y = W_L x_y) and W_L^T f_ext is cached,
    // so only the cubature rows of W_L are read again.
    {
        Phase p(ctx, DAE_PHASE_WTA, (gram && !gout) ? 2 : 1);
        if (gram && !gout) launch_xy(s, w.X[(L - 1) & 1], top.ld, K, r, w.zvec, P.h, w.xy, ns);
        launch_wta(s, wa);
    }
    int in_ncol = 1, cur = 0;
    const bool tc_rev = d->prec != DAE_FP32 && d->layers[0].tmR_ok;
    if (tc_rev) {
        // complex-step reverse pass on the tensor cores: delta_l = W_l^T g_l, the epilogue
        // forms g_{l-1} (complex act' of the layer below) as the next B operand
        const int ob = out_bf16_of(d->prec);
        const int of32 = (d->prec == DAE_TF32) ? 2 : 0;
        {
            BwdArgs ba;
            memset(&ba, 0, sizeof ba);
            ba.n_o = d->widths[L - 1]; ba.r = r;
            ba.in_part = w.bwd_part[0]; ba.in_split = in_split; ba.in_ncol = 1;
            ba.S1 = w.S1[L - 2]; ba.T = w.T[L - 2]; ba.ns = ns;
            Phase p(ctx, DAE_PHASE_BWD, 1);
            launch_bwd_prep_tc(s, ba, w.Cb, d->layers[L - 2].ldT, w.G32[0], w.Gh[0], w.Gl[0], of32, ob);
        }
        if (w.chain_ok) {
            ChainLaunch cl = {};
            cl.jobs = w.rev_jobs; cl.n_jobs = L - 1; cl.Cp = w.Cb; cl.grid = ctx->sm_count;
            cl.gb = w.gbar; cl.ns = ns; cl.status = ctx->d_status; cl.split_part = w.chain_part;
            cl.split_cnt = w.chain_cnt;
            Phase p(ctx, DAE_PHASE_BWD, 1);
            if (!launch_chain(s, cl, d->prec))
                return fail(ctx, DAE_ERR_CUDA, "reverse layer-chain launch failed");
        } else {
            for (int l = L - 2; l >= 0; --l) {
                FwdArgs a;
                fill_rev_args(d, l, a);
                a.ns = ns;
                a.status = ctx->d_status;
                Phase p(ctx, DAE_PHASE_BWD, 1);
                if (!launch_fwd_tc(s, a, d->prec, sm))
                    return fail(ctx, DAE_ERR_UNSUPPORTED, "reverse GEMM launch failed for layer %d", l);
            }
        }
        cur = 1;
        in_split = 1;
    } else {
    for (int l = L - 2; l >= 0; --l) {
        BwdArgs ba;
        ba.W = d->layers[l].W; ba.ld = d->layers[l].ld;
        ba.n_o = d->widths[l + 1]; ba.n_i = d->widths[l]; ba.r = r;
        ba.in_part = w.bwd_part[cur]; ba.in_split = in_split; ba.in_ncol = in_ncol;
        ba.S1 = w.S1[l]; ba.T = w.T[l]; ba.g = w.gbuf;
        ba.out_split = bwd_split(ba.n_i, ba.n_o, sm);
        ba.out_part = w.bwd_part[cur ^ 1];
        ba.ns = ns;
        {
            Phase p(ctx, DAE_PHASE_BWD, 2);
            launch_bwd(s, ba);
        }
        cur ^= 1;
        in_split = ba.out_split;
        in_ncol = 1 + r;
    }
    }
    aa.bwd_part = w.bwd_part[cur]; aa.bwd_split = in_split;
    {
        Phase p(ctx, DAE_PHASE_ASSEMBLE, 1);
        launch_control(s, aa);
    }
    CU(ctx, cudaGetLastError());
    return DAE_OK;
}

dae_status ensure_frames(dae_decoder* d, int n_frames) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (!w.rc) {
        TRY(dmalloc(ctx, &w.rc, 1));
        TRY(dmalloc(ctx, &w.qout, (size_t)(d->np + d->r)));
    }
    if (n_frames > w.hist_cap) {
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.hist);
        dfree(w.traj);
        const int cap = std::max(n_frames, 16);
        TRY(dmalloc(ctx, &w.hist, (size_t)cap));
        TRY(dmalloc(ctx, &w.traj, (size_t)cap * (d->np + d->r)));
        w.hist_cap = cap;
        w.graph_ok = false;
    }
    return DAE_OK;
}

void drop_graph(Workspace& w) {
    if (w.gexec) cudaGraphExecDestroy(w.gexec);
    w.gexec = nullptr;
    w.graph_ok = false;
}

// Add a WHILE conditional node to g after dep (may be null); returns its body graph.
dae_status add_while(dae_ctx* ctx, cudaGraph_t g, cudaGraphNode_t* dep,
                     cudaGraphConditionalHandle h, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    CU(ctx, cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &p));
    *body = p.conditional.phGraph_out[0];
    return DAE_OK;
}

dae_status sole_sink(dae_ctx* ctx, cudaGraph_t g, cudaGraphNode_t* out) {
    size_t n = 0;
    CU(ctx, cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    CU(ctx, cudaGraphGetNodes(g, nodes.data(), &n));
    for (auto nd : nodes) {
        size_t nout = 0;
        CU(ctx, cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout));
        if (nout == 0) { *out = nd; return DAE_OK; }
    }
    return fail(ctx, DAE_ERR_CUDA, "graph has no sink node");
}

// Capture: init -> WHILE(frames) { frame_start -> WHILE(evals) { evaluation } -> frame_finish }
dae_status build_graph(dae_decoder* d, const dae_mesh* m, EvalParams P) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    drop_graph(w);
    // capture on a private stream (the caller's stream may be the legacy default stream,
    // which cannot be captured); the executable graph is launched on the caller's stream
    if (!ctx->cap_stream) CU(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    const cudaStream_t saved_stream = ctx->stream;
    ctx->stream = ctx->cap_stream;
    cudaStream_t s = ctx->cap_stream;
    const unsigned saved_prof = ctx->prof_on;
    ctx->prof_on = 0;
    cudaGraph_t g = nullptr;
    CU(ctx, cudaGraphCreate(&g, 0));
    dae_status st = DAE_OK;
    const int r = d->np + d->r;   // system size
    do {
        cudaGraphConditionalHandle hout, hin;
        if (cudaGraphConditionalHandleCreate(&hout, g, 0, 0) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        if (cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        launch_roll_init(s, w.rc, hout, 1, ctx->d_kcount);
        if (cudaStreamEndCapture(s, &g) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        cudaGraphNode_t a, outer, sn, inner;
        if ((st = sole_sink(ctx, g, &a))) break;
        cudaGraph_t bo, bi;
        if ((st = add_while(ctx, g, &a, hout, &outer, &bo))) break;
        if (cudaGraphConditionalHandleCreate(&hin, bo, 0, 0) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        if (cudaStreamBeginCaptureToGraph(s, bo, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        launch_frame_start(s, w.rc, w.ns, w.qbar, w.qbar_dot, P.dt, r, hin, 1, ctx->d_kcount);
        if (cudaStreamEndCapture(s, &bo) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        if ((st = sole_sink(ctx, bo, &sn))) break;
        if ((st = add_while(ctx, bo, &sn, hin, &inner, &bi))) break;
        // evaluation body
        if (cudaStreamBeginCaptureToGraph(s, bi, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        const long long l0 = ctx->launches;
        P.hcond = hin; P.use_cond = 1; P.kcount = ctx->d_kcount;
        dae_status es = enqueue_eval(d, m, w.ns, nullptr, P);
        const int kpe = (int)(ctx->launches - l0);
        ctx->launches = l0;
        cudaGraph_t bi2 = bi;
        cudaError_t ce = cudaStreamEndCapture(s, &bi2);
        if (es) { st = es; break; }
        if (ce != cudaSuccess) { st = fail(ctx, DAE_ERR_CUDA, "capture failed: %s", cudaGetErrorString(ce)); break; }
        w.kpe = kpe;
        if (cudaStreamBeginCaptureToGraph(s, bo, &inner, nullptr, 1, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        launch_frame_finish(s, w.rc, w.ns, w.qbar, w.qbar_dot, P.dt, r, w.traj, w.hist, w.qout, hout,
                            1, ctx->d_kcount);
        if (cudaStreamEndCapture(s, &bo) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        cudaError_t ie = cudaGraphInstantiate(&w.gexec, g, 0);
        if (ie != cudaSuccess) { st = fail(ctx, DAE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie)); break; }
    } while (0);
    ctx->prof_on = saved_prof;
    ctx->stream = saved_stream;
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (st) {
        if (ctx->err.empty()) fail(ctx, st, "frame graph construction failed");
        w.gexec = nullptr;
        return st;
    }
    w.graph_ok = true;
    return DAE_OK;
}

// Run n_frames implicit-Euler frames on the device (Newton evaluations until the
// device control marks each frame done).  The kernels executed per evaluation are
// patched into the counter by k_control when the kpe field is known, so the graph
// needs it at capture time: captured with kpe from a dry count.
dae_status run_frames(dae_decoder* d, const dae_mesh* m, EvalParams P, int n_frames, int given_q0,
                      int advance, const double* q_in_dev) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    cudaStream_t s = ctx->stream;
    const int r = d->np + d->r;   // system size
    TRY(ensure_frames(d, n_frames));
    ctx->launches += 1;
    launch_roll_setup(s, w.rc, n_frames, given_q0, advance, q_in_dev, r);
    if (ctx->prof_on) {
        // explicit launches, host checks each frame's done flag after every evaluation
        drop_graph(w);
        ctx->launches += 1;
        launch_roll_init(s, w.rc, 0, 0, nullptr);
        for (int f = 0; f < n_frames; ++f) {
            ctx->launches += 1;
            launch_frame_start(s, w.rc, w.ns, w.qbar, w.qbar_dot, P.dt, r, 0, 0, nullptr);
            for (int e = 0; e < P.opts->max_evals; ++e) {
                TRY(enqueue_eval(d, m, w.ns, nullptr, P));
                int done = 0;
                CU(ctx, cudaMemcpyAsync(&done, &w.ns->done, sizeof(int), cudaMemcpyDeviceToHost, s));
                CU(ctx, cudaStreamSynchronize(s));
                if (done) break;
            }
            ctx->launches += 1;
            launch_frame_finish(s, w.rc, w.ns, w.qbar, w.qbar_dot, P.dt, r, w.traj, w.hist, w.qout,
                                0, 0, nullptr);
        }
        CU(ctx, cudaGetLastError());
        return DAE_OK;
    }
    GraphKey key;
    memset(&key, 0, sizeof key);
    key.mesh_id = m->id; key.dec_id = d->id; key.cub_w = P.cub_w; key.cub_tets = P.cub_tets; key.fe_w = w.fe_w;
    key.hist = w.hist; key.traj = w.traj; key.fext = P.f_ext; key.n_cub = P.n_cub;
    key.gram = w.G && w.G_mesh == m->id; key.prec = d->prec;
    key.max_iter = P.opts->max_iter; key.max_halvings = P.opts->max_halvings;
    key.max_evals = P.opts->max_evals; key.dt = P.dt; key.h = P.h; key.tol = P.opts->tol;
    key.c_armijo = P.opts->c_armijo; key.max_step = P.opts->max_step;
    key.xtol = P.opts->xtol;
    key.gs = w.gs_ok ? (w.Gs32 ? (const void*)w.Gs32 : (const void*)w.Gsh) : nullptr;
    key.wn = P.wnet ? (const void*)w.wn_B1 : nullptr;
    key.gram = (key.gram ? 1 : 0) | (gram_out(d, m) ? 2 : 0);
    if (!w.graph_ok || memcmp(&key, &w.gkey, sizeof key) != 0) {
        // kernels per evaluation: count once with a dry capture so k_control can add them
        P.kpe = 0;
        TRY(build_graph(d, m, P));
        P.kpe = w.kpe;
        TRY(build_graph(d, m, P));
        w.gkey = key;
    }
    CU(ctx, cudaGraphLaunch(w.gexec, s));
    return DAE_OK;
}

dae_status check_common(dae_ctx* ctx, const dae_decoder* dec, const dae_mesh* m) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    if (!dec || dec->ctx != ctx) return fail(ctx, DAE_ERR_INVALID_ARG, "decoder missing or from another context");
    if (dec->ws.sync_epoch != ctx->timeout_epoch) {
        // zero the layer-chain synchronisation state after a timed-out launch
        Workspace& w = const_cast<dae_decoder*>(dec)->ws;
        CU(ctx, cudaSetDevice(ctx->device));
        if (w.gbar) CU(ctx, cudaMemsetAsync(w.gbar, 0, sizeof(GridBar), ctx->stream));
        if (w.chain_cnt) CU(ctx, cudaMemsetAsync(w.chain_cnt, 0, w.chain_cnt_n * sizeof(unsigned), ctx->stream));
        w.sync_epoch = ctx->timeout_epoch;
    }
    if (m) {
        if (m->ctx != ctx) return fail(ctx, DAE_ERR_INVALID_ARG, "mesh from another context");
        if (3 * m->n_vert != dec->N)
            return fail(ctx, DAE_ERR_INVALID_ARG, "decoder output %d != 3 x %d mesh vertices", dec->N, m->n_vert);
    }
    CU(ctx, cudaSetDevice(ctx->device));
    return DAE_OK;
}

void to_report(const NewtonState& s, dae_newton_report* rep) {
    rep->iters = s.iters;
    rep->evals = s.evals;
    rep->converged = s.converged;
    rep->status = s.status;
    rep->phi_norm0 = s.phi_norm0;
    rep->phi_norm = std::sqrt(s.merit_acc);
    rep->energy = s.energy;
    rep->alpha = s.alpha;
    rep->full_evals = s.nfull;
}

void fill_opts(const dae_newton_opts* in, dae_newton_opts* o) {
    dae_default_newton_opts(o);
    if (in) *o = *in;
    if (o->max_evals <= 0) o->max_evals = o->max_iter + 3;
    if (o->h_cs <= 0) o->h_cs = std::ldexp(1.0, -20);
}

dae_status stage_cubature(dae_decoder* d, Stage& st, int n_cub, const int* cub_tets,
                          const float* cub_w, int n_w, const int** dt_out, const float** dw_out) {
    TRY(ensure_cubature(d, n_cub, n_w));
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    if (n_cub > 0) {
        CU(ctx, cudaMemcpyAsync(w.cub_tets, cub_tets, (size_t)n_cub * sizeof(int),
                                cudaMemcpyDefault, ctx->stream));
        if (cub_w)
            CU(ctx, cudaMemcpyAsync(w.cub_w, cub_w, (size_t)n_w * sizeof(float), cudaMemcpyDefault,
                                    ctx->stream));
    }
    *dt_out = w.cub_tets;
    *dw_out = w.cub_w;
    if (!cub_w && n_cub > 0) {
        // weights predicted by the attached weight network (one set per frame)
        if (w.wn_cap < n_cub) {
            dfree(w.wn_w);
            TRY(dmalloc(ctx, &w.wn_w, (size_t)n_cub));
            w.wn_cap = n_cub;
            w.graph_ok = false;
        }
        *dw_out = w.wn_w;
    }
    (void)st;
    return DAE_OK;
}

dae_status stage_fext(dae_decoder* d, const float* f_ext, const float** out) {
    dae_ctx* ctx = d->ctx;
    if (!f_ext) {
        *out = nullptr;
        return DAE_OK;
    }
    CU(ctx, cudaMemcpyAsync(d->ws.f_ext, f_ext, (size_t)d->N * sizeof(float), cudaMemcpyDefault,
                            ctx->stream));
    *out = d->ws.f_ext;
    return DAE_OK;
}

dae_status validate_cub(dae_ctx* ctx, const dae_mesh* m, int n_cub, const int* cub_tets,
                        const float* cub_w, const dae_decoder* d = nullptr) {
    if (n_cub < 0) return fail(ctx, DAE_ERR_INVALID_ARG, "n_cub < 0");
    if (n_cub > 0 && !cub_tets) return fail(ctx, DAE_ERR_INVALID_ARG, "cubature tets missing");
    if (n_cub > 0 && !cub_w && !(d && d->ws.wn_B1))
        return fail(ctx, DAE_ERR_INVALID_ARG, "cubature weights missing (and no weight network attached)");
    if (d && d->ws.wn_B1 && !cub_w && d->ws.wn_ntet != m->n_tet)
        return fail(ctx, DAE_ERR_INVALID_ARG, "weight network has %d outputs for %d elements",
                    d->ws.wn_ntet, m->n_tet);
    if (n_cub > 0 && !on_device(cub_tets)) {
        for (int i = 0; i < n_cub; ++i)
            if (cub_tets[i] < 0 || cub_tets[i] >= m->n_tet)
                return fail(ctx, DAE_ERR_INVALID_ARG, "cubature tet %d out of range", cub_tets[i]);
    }
    return DAE_OK;
}

// ------------------------------------------------------- batched systems --
// One Newton step of many independent systems (dae_newton_step_batched): every
// kernel of an evaluation runs once for all systems (grouped launches), inside one
// graph whose evaluation loop runs while any system is not done.
struct BatchKey {
    unsigned long long dec_id, mesh_id;
    const void* cub_tets; const void* cub_w; const void* fe_w; const void* G; const void* pext;
    const void* gs; const void* wn;
    int n_cub, has_fext;
};

// Ties between the domains of one grouped step (dae_newton_step_coupled): the topology
// on the host and its device arrays.
struct Coupling {
    int n_dom = 0, n_tv = 0, n_tot = 0, n_comp = 0;
    std::vector<int> pairs, anchors;   // as given (cache key)
    double kc = 0;
    std::vector<int> off, ntv_dom, tv_dom, tv_vert, tv_slot, nb_off, nb, n_anch, dtv_off, dtv,
        unk_dom, comp_off, order, parent, cp_off, cp;
    char* dev = nullptr;               // one allocation: arguments and arrays
    CoupledArgs* args = nullptr;       // device
    CoupledState* cs = nullptr;        // device
    ~Coupling() { if (dev) cudaFree(dev); }
};

// Tie vertices, neighbour lists, the domain forest (a pair joins a child domain to its
// parent; the lowest domain of each connected component is its root) and its post-order.
dae_status build_topology(dae_ctx* ctx, Coupling& c, const std::vector<int>& r,
                          const std::vector<int>& n_vert, int n_pairs, const int* pairs,
                          int n_anch, const int* anch) {
    const int D = (int)r.size();
    c.n_dom = D;
    c.pairs.assign(pairs, pairs + 4 * (size_t)n_pairs);
    c.anchors.assign(anch, anch + 2 * (size_t)n_anch);
    c.off.assign(D + 1, 0);
    for (int d = 0; d < D; ++d) c.off[d + 1] = c.off[d] + r[d];
    c.n_tot = c.off[D];
    c.unk_dom.resize(c.n_tot);
    for (int d = 0; d < D; ++d)
        for (int i = c.off[d]; i < c.off[d + 1]; ++i) c.unk_dom[i] = d;
    std::map<std::pair<int, int>, int> tv;
    auto tie = [&](int d, int v) -> int {
        auto it = tv.find({d, v});
        if (it != tv.end()) return it->second;
        const int t = (int)c.tv_dom.size();
        tv[{d, v}] = t;
        c.tv_dom.push_back(d);
        c.tv_vert.push_back(v);
        return t;
    };
    auto bad_vertex = [&](int d, int v) { return d < 0 || d >= D || v < 0 || v >= n_vert[d]; };
    std::vector<std::vector<int>> nbl;
    std::vector<std::pair<int, int>> ptv(n_pairs);
    for (int p = 0; p < n_pairs; ++p) {
        const int d = pairs[4 * p], i = pairs[4 * p + 1], e = pairs[4 * p + 2], j = pairs[4 * p + 3];
        if (bad_vertex(d, i) || bad_vertex(e, j))
            return fail(ctx, DAE_ERR_INVALID_ARG, "tie pair %d: domain or vertex out of range", p);
        if (d == e) return fail(ctx, DAE_ERR_INVALID_ARG, "tie pair %d joins a domain to itself", p);
        ptv[p] = {tie(d, i), tie(e, j)};
    }
    std::vector<int> at(n_anch);
    for (int a = 0; a < n_anch; ++a) {
        if (bad_vertex(anch[2 * a], anch[2 * a + 1]))
            return fail(ctx, DAE_ERR_INVALID_ARG, "anchor %d: domain or vertex out of range", a);
        at[a] = tie(anch[2 * a], anch[2 * a + 1]);
    }
    c.n_tv = (int)c.tv_dom.size();
    nbl.assign(c.n_tv, {});
    for (auto& p : ptv) { nbl[p.first].push_back(p.second); nbl[p.second].push_back(p.first); }
    c.n_anch.assign(c.n_tv, 0);
    for (int t : at) c.n_anch[t] += 1;
    c.nb_off.assign(c.n_tv + 1, 0);
    c.nb.clear();
    for (int t = 0; t < c.n_tv; ++t) {
        c.nb.insert(c.nb.end(), nbl[t].begin(), nbl[t].end());
        c.nb_off[t + 1] = (int)c.nb.size();
    }
    // each domain's tie vertices (slot = position in its list)
    c.ntv_dom.assign(D, 0);
    c.tv_slot.assign(c.n_tv, 0);
    c.dtv_off.assign(D + 1, 0);
    std::vector<std::vector<int>> dl(D);
    for (int t = 0; t < c.n_tv; ++t) { c.tv_slot[t] = (int)dl[c.tv_dom[t]].size(); dl[c.tv_dom[t]].push_back(t); }
    c.dtv.clear();
    for (int d = 0; d < D; ++d) {
        c.ntv_dom[d] = (int)dl[d].size();
        c.dtv.insert(c.dtv.end(), dl[d].begin(), dl[d].end());
        c.dtv_off[d + 1] = (int)c.dtv.size();
    }
    // the domain graph must be a forest
    std::vector<int> uf(D);
    for (int d = 0; d < D; ++d) uf[d] = d;
    std::function<int(int)> find = [&](int x) { return uf[x] == x ? x : (uf[x] = find(uf[x])); };
    std::set<std::pair<int, int>> edges;
    for (auto& p : ptv) {
        const int a = c.tv_dom[p.first], b = c.tv_dom[p.second];
        edges.insert({std::min(a, b), std::max(a, b)});
    }
    std::vector<std::vector<int>> adj(D);
    for (auto& e : edges) {
        const int a = find(e.first), b = find(e.second);
        if (a == b) return fail(ctx, DAE_ERR_UNSUPPORTED, "the ties' domain graph has a cycle (a forest is required)");
        uf[a] = b;
        adj[e.first].push_back(e.second);
        adj[e.second].push_back(e.first);
    }
    // components: root = lowest domain; iterative DFS for parents and post-order
    c.parent.assign(D, -2);
    c.comp_off.assign(1, 0);
    c.order.clear();
    for (int root = 0; root < D; ++root) {
        if (c.parent[root] != -2) continue;
        c.parent[root] = -1;
        std::vector<std::pair<int, size_t>> st{{root, 0}};
        while (!st.empty()) {
            auto& top = st.back();
            const int d = top.first;
            if (top.second < adj[d].size()) {
                const int e = adj[d][top.second++];
                if (c.parent[e] == -2) { c.parent[e] = d; st.push_back({e, 0}); }
            } else {
                c.order.push_back(d);
                st.pop_back();
            }
        }
        c.comp_off.push_back((int)c.order.size());
    }
    c.n_comp = (int)c.comp_off.size() - 1;
    // the pairs of each child with its parent: (tie vertex in the child, in the parent)
    std::vector<std::vector<int>> cpl(D);
    for (auto& p : ptv) {
        int a = p.first, b = p.second;
        if (c.parent[c.tv_dom[a]] != c.tv_dom[b]) std::swap(a, b);
        cpl[c.tv_dom[a]].push_back(a);
        cpl[c.tv_dom[a]].push_back(b);
    }
    c.cp_off.assign(D + 1, 0);
    c.cp.clear();
    for (int d = 0; d < D; ++d) {
        c.cp.insert(c.cp.end(), cpl[d].begin(), cpl[d].end());
        c.cp_off[d + 1] = (int)(c.cp.size() / 2);
    }
    return DAE_OK;
}

struct BatchPlan {
    std::vector<BatchKey> key;
    double dt = 0;
    dae_newton_opts opts;
    int prec = -1;
    int n = 0;
    unsigned long long epoch = 0;
    // device argument arrays (one allocation)
    char* dev = nullptr;
    SeedArgs* seed = nullptr; CubArgs* cub = nullptr; XyArgs* xy = nullptr; WtaArgs* wta = nullptr;
    PrepArgs* prep = nullptr; ColsumArgs* cs = nullptr; DsumArgs* ds = nullptr; CtlArgs* ctl = nullptr;
    FrameArgs* frame = nullptr;
    GatherArgs* gather = nullptr; int max_gather = 0;
    WnetArgs* wnet = nullptr; int max_wn_H1 = 0, max_wn_n = 0;   // predicted weights
    LinArgs* lin = nullptr; int max_lin_blocks = 0;               // linear subspaces
    double* q0 = nullptr; double* qout = nullptr;   // [n][kMaxR]
    NewtonState* ns_out = nullptr;                  // [n] report copies
    ChainJob* jobs = nullptr; int* stage_off = nullptr;
    GridBar* gb = nullptr;
    int* flag = nullptr;            // any system still iterating (explicit launches)
    struct Chain { size_t job0; size_t st0; int n_stages; int Cp; };
    std::vector<Chain> fwd, rev;
    int max_elems = 0, max_cub = 0, max_K = 0, max_splits = 1, max_ld = 0, max_ent = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t staged = nullptr;   // host staging buffer free again
    Coupling* cpl = nullptr;        // ties between the systems (dae_newton_step_coupled)
};

void free_batch(dae_ctx* ctx) {
    for (void** slot : {&ctx->batch, &ctx->batch_coupled}) {
        BatchPlan* b = (BatchPlan*)*slot;
        if (!b) continue;
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->dev) cudaFree(b->dev);
        if (b->staged) cudaEventDestroy(b->staged);
        delete b->cpl;
        delete b;
        *slot = nullptr;
    }
}

// Device copy of a coupling's topology and state, with the domains' records.
dae_status upload_coupling(dae_ctx* ctx, Coupling& c, const std::vector<TieDom>& dom, double dt,
                           double h, const dae_newton_opts& o) {
    if (c.dev) cudaFree(c.dev);
    c.dev = nullptr;
    const int D = c.n_dom;
    size_t off = 0;
    auto place = [&](size_t bytes) { const size_t q = off; off += round_up(std::max(bytes, (size_t)16), 256); return q; };
    auto ints = [&](const std::vector<int>& v) { return place(v.size() * sizeof(int)); };
    const size_t o_args = place(sizeof(CoupledArgs)), o_cs = place(sizeof(CoupledState));
    const size_t o_dom = place(D * sizeof(TieDom));
    const size_t o_unk = ints(c.unk_dom), o_dtvo = ints(c.dtv_off), o_dtv = ints(c.dtv);
    const size_t o_tvd = ints(c.tv_dom), o_tvv = ints(c.tv_vert), o_tvs = ints(c.tv_slot);
    const size_t o_nbo = ints(c.nb_off), o_nb = ints(c.nb), o_na = ints(c.n_anch);
    const size_t o_co = ints(c.comp_off), o_ord = ints(c.order), o_par = ints(c.parent);
    const size_t o_cpo = ints(c.cp_off), o_cp = ints(c.cp);
    const size_t o_uj = place((size_t)c.n_tv * 3 * (1 + kMaxR) * sizeof(float));
    const size_t o_g = place((size_t)c.n_tv * 3 * sizeof(double));
    const size_t o_q = place((size_t)4 * c.n_tot * sizeof(double));
    const size_t o_S = place((size_t)D * kMaxR * kMaxR * sizeof(double));
    const size_t o_X = place((size_t)D * kMaxR * kMaxR * sizeof(double));
    const size_t o_y = place((size_t)D * kMaxR * sizeof(double));
    CU(ctx, cudaMalloc(&c.dev, off));
    CU(ctx, cudaMemset(c.dev, 0, off));
    char* B = c.dev;
    auto put = [&](size_t o_, const std::vector<int>& v) {
        return v.empty() ? cudaSuccess : cudaMemcpy(B + o_, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
    };
    CoupledArgs a;
    memset(&a, 0, sizeof a);
    a.n_dom = D; a.n_tv = c.n_tv; a.n_tot = c.n_tot;
    a.dom = (const TieDom*)(B + o_dom);
    a.unk_dom = (const int*)(B + o_unk); a.dtv_off = (const int*)(B + o_dtvo); a.dtv = (const int*)(B + o_dtv);
    a.tv_dom = (const int*)(B + o_tvd); a.tv_vert = (const int*)(B + o_tvv); a.tv_slot = (const int*)(B + o_tvs);
    a.nb_off = (const int*)(B + o_nbo); a.nb = (const int*)(B + o_nb); a.n_anch = (const int*)(B + o_na);
    a.uJ = (float*)(B + o_uj); a.g = (double*)(B + o_g);
    a.kc = c.kc; a.dt = dt; a.h = h;
    a.cs = (CoupledState*)(B + o_cs);
    double* q = (double*)(B + o_q);
    a.q_acc = q; a.q_trial = q + c.n_tot; a.delta = q + 2 * c.n_tot; a.phi = q + 3 * c.n_tot;
    a.tol = o.tol; a.c_armijo = o.c_armijo; a.max_step = o.max_step; a.xtol = o.xtol;
    a.max_iter = o.max_iter; a.max_halvings = o.max_halvings; a.max_evals = o.max_evals;
    a.n_comp = c.n_comp; a.comp_off = (const int*)(B + o_co); a.order = (const int*)(B + o_ord);
    a.parent = (const int*)(B + o_par); a.cp_off = (const int*)(B + o_cpo); a.cp = (const int*)(B + o_cp);
    a.S = (double*)(B + o_S); a.X = (double*)(B + o_X); a.y = (double*)(B + o_y);
    cudaError_t e = cudaMemcpy(B + o_args, &a, sizeof a, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B + o_dom, dom.data(), D * sizeof(TieDom), cudaMemcpyHostToDevice);
    for (auto pr : {std::make_pair(o_unk, &c.unk_dom), std::make_pair(o_dtvo, &c.dtv_off),
                    std::make_pair(o_dtv, &c.dtv), std::make_pair(o_tvd, &c.tv_dom),
                    std::make_pair(o_tvv, &c.tv_vert), std::make_pair(o_tvs, &c.tv_slot),
                    std::make_pair(o_nbo, &c.nb_off), std::make_pair(o_nb, &c.nb),
                    std::make_pair(o_na, &c.n_anch), std::make_pair(o_co, &c.comp_off),
                    std::make_pair(o_ord, &c.order), std::make_pair(o_par, &c.parent),
                    std::make_pair(o_cpo, &c.cp_off), std::make_pair(o_cp, &c.cp)})
        if (e == cudaSuccess) e = put(pr.first, *pr.second);
    if (e != cudaSuccess) return fail(ctx, DAE_ERR_CUDA, "coupling upload: %s", cudaGetErrorString(e));
    c.args = (CoupledArgs*)(B + o_args);
    c.cs = a.cs;
    return DAE_OK;
}

dae_status ensure_pinned(dae_ctx* ctx, size_t bytes) {
    if (ctx->pinned_bytes >= bytes) return DAE_OK;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    const size_t nb = std::max(bytes, (size_t)1 << 20);
    CU(ctx, cudaHostAlloc(&ctx->pinned, nb, cudaHostAllocDefault));
    ctx->pinned_bytes = nb;
    return DAE_OK;
}

// Grouped chain launches: stage t of a chain holds layer t (forward) or reverse job t
// of each system of a group of at most kMaxGroupJobs systems.  B-operand maps are
// re-encoded with the launch's column count as box height (rows past a system's own
// columns read as zero).
dae_status batch_chain_jobs(dae_ctx* ctx, const std::vector<dae_decoder*>& ds, bool fwd,
                            const std::vector<Outs>& outs, double dt, double h,
                            std::vector<ChainJob>& jobs, std::vector<int>& stage_off,
                            std::vector<BatchPlan::Chain>& chains) {
    const int n = (int)ds.size();
    for (int g0 = 0; g0 < n; g0 += kMaxGroupJobs) {
        const int g1 = std::min(n, g0 + kMaxGroupJobs);
        int CP = 16, n_st = 0;
        for (int i = g0; i < g1; ++i) {
            CP = std::max(CP, fwd ? ds[i]->ws.Cp : ds[i]->ws.Cb);
            n_st = std::max(n_st, fwd ? ds[i]->L : ds[i]->L - 1);
        }
        if (CP > 112) return fail(ctx, DAE_ERR_UNSUPPORTED, "column count %d too large", CP);
        BatchPlan::Chain c;
        c.job0 = jobs.size();
        c.st0 = stage_off.size();
        c.n_stages = n_st;
        c.Cp = CP;
        for (int t = 0; t < n_st; ++t) {
            stage_off.push_back((int)(jobs.size() - c.job0));
            int base = 0;
            for (int i = g0; i < g1; ++i) {
                const dae_decoder* d = ds[i];
                const Workspace& w = d->ws;
                const int L = d->L;
                ChainJob j;
                if (fwd) {
                    if (t >= L) continue;
                    if (t == L - 1) make_out_job(d, outs[i], dt, h, j);
                    else make_fwd_job(d, t, j);
                    if (w.Cp != CP) {
                        const Layer& ly = d->layers[t];
                        const bool f32 = d->prec == DAE_TF32;
                        const int buf = t & 1;
                        bool ok = make_tmap(&j.tm[2], f32 ? (const void*)w.X[buf] : (const void*)w.Xh[buf],
                                            f32, ly.ld, w.Cp, CP);
                        if (d->prec == DAE_BF16X3) ok = ok && make_tmap(&j.tm[3], w.Xl[buf], false, ly.ld, w.Cp, CP);
                        else j.tm[3] = j.tm[2];
                        if (!ok) return fail(ctx, DAE_ERR_UNSUPPORTED, "tensor map encoding failed");
                    }
                } else {
                    if (t >= L - 1) continue;
                    const int l = L - 2 - t;
                    make_rev_job(d, l, j);
                    if (w.Cb != CP) {
                        const Layer& ly = d->layers[l];
                        const bool f32 = d->prec == DAE_TF32;
                        const int gb = (L - 2 - l) & 1;
                        bool ok = make_tmap(&j.tm[2], f32 ? (const void*)w.G32[gb] : (const void*)w.Gh[gb],
                                            f32, ly.ldT, w.Cb, CP);
                        if (d->prec == DAE_BF16X3) ok = ok && make_tmap(&j.tm[3], w.Gl[gb], false, ly.ldT, w.Cb, CP);
                        else j.tm[3] = j.tm[2];
                        if (!ok) return fail(ctx, DAE_ERR_UNSUPPORTED, "tensor map encoding failed");
                    }
                }
                j.a.ns = w.ns;
                j.item_base = base;
                base += j.tiles;
                jobs.push_back(j);
            }
        }
        stage_off.push_back((int)(jobs.size() - c.job0));
        chains.push_back(c);
    }
    return DAE_OK;
}

// One Newton evaluation of every system still iterating, on ctx->stream (inside a
// capture or as explicit launches), ending with the kernel that sets the loop condition
// (hc) or writes the any-running flag.
dae_status enqueue_batch_eval(dae_ctx* ctx, const BatchPlan* b, dae_prec prec,
                              cudaGraphConditionalHandle hc, int* flag) {
    cudaStream_t s = ctx->stream;
    const int n = b->n;
    {
        Phase p(ctx, DAE_PHASE_SEED, 1);
        launch_seed_batched(s, b->seed, n, b->max_elems);
    }
    for (const auto& c : b->fwd) {
        ChainLaunch cl = {};
        cl.jobs = b->jobs + c.job0; cl.n_jobs = 0; cl.Cp = c.Cp; cl.grid = ctx->sm_count;
        cl.gb = b->gb; cl.status = ctx->d_status;
        cl.stage_off = b->stage_off + c.st0; cl.n_stages = c.n_stages;
        Phase p(ctx, DAE_PHASE_FWD_OUT, 1);
        if (!launch_chain(s, cl, prec)) return fail(ctx, DAE_ERR_CUDA, "grouped chain launch failed");
    }
    if (b->max_wn_H1 > 0) {
        Phase p(ctx, DAE_PHASE_CUBATURE, 3);
        launch_wnet_batched(s, b->wnet, n, b->max_wn_H1, b->max_wn_n);
    }
    if (b->max_lin_blocks > 0) {
        Phase p(ctx, DAE_PHASE_CUBATURE, 1);
        launch_linear_batched(s, b->lin, n, b->max_lin_blocks);
    }
    {
        Phase p(ctx, DAE_PHASE_CUBATURE, 1);
        launch_cubature_batched(s, b->cub, n, b->max_cub);
    }
    if (b->cpl) {
        // u and J at the tie vertices (from the output layer's input activations)
        Phase p(ctx, DAE_PHASE_CUBATURE, 1);
        launch_tie_uj(s, b->cpl->args, b->cpl->n_tv);
    }
    {
        // phi and the decisions: systems whose iterate starts no new Newton step skip the
        // reverse pass below (coupled: every domain's phi, then one global decision)
        Phase p(ctx, DAE_PHASE_ASSEMBLE, b->cpl ? 4 : 3);
        launch_decide_batched(s, b->cs, b->ds, b->ctl, n, b->max_ent);
        if (b->cpl) launch_coupled_decide(s, b->cpl->args);
    }
    {
        Phase p(ctx, DAE_PHASE_WTA, 2);
        launch_xy_batched(s, b->xy, n, b->max_K);
        launch_wta_batched(s, b->wta, n, b->max_K, b->max_splits);
    }
    {
        Phase p(ctx, DAE_PHASE_BWD, 1);
        launch_bwd_prep_tc_batched(s, b->prep, n, b->max_ld);
    }
    for (const auto& c : b->rev) {
        ChainLaunch cl = {};
        cl.jobs = b->jobs + c.job0; cl.n_jobs = 0; cl.Cp = c.Cp; cl.grid = ctx->sm_count;
        cl.gb = b->gb; cl.status = ctx->d_status;
        cl.stage_off = b->stage_off + c.st0; cl.n_stages = c.n_stages;
        Phase p(ctx, DAE_PHASE_BWD, 1);
        if (!launch_chain(s, cl, prec)) return fail(ctx, DAE_ERR_CUDA, "grouped chain launch failed");
    }
    {
        Phase p(ctx, DAE_PHASE_ASSEMBLE, b->cpl ? 4 : 2);
        launch_control_batched(s, b->ctl, n);
        if (b->cpl) {
            // the global Newton step over the domain forest, then the next trial
            launch_coupled_solve(s, b->cpl->args, b->cpl->n_comp);
            launch_coupled_update(s, b->cpl->args);
        }
        launch_batch_cond(s, b->frame, n, hc, flag);
    }
    CU(ctx, cudaGetLastError());
    return DAE_OK;
}

// Argument arrays, chain jobs and the graph of one batch (cached while the systems'
// decoders, meshes, staging buffers and the options stay the same).
dae_status build_batch(dae_ctx* ctx, BatchPlan* b, const std::vector<dae_decoder*>& ds,
                       const std::vector<const dae_mesh*>& ms, const std::vector<int>& ncub,
                       const std::vector<int>& hasf, const std::vector<int>& pred, double dt,
                       const dae_newton_opts& opts) {
    const int n = (int)ds.size();
    Coupling* cpl = b->cpl;
    std::vector<TieDom> tdom(cpl ? n : 0);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    if (b->dev) cudaFree(b->dev);
    b->dev = nullptr;
    b->fwd.clear();
    b->rev.clear();
    const double h = opts.h_cs;
    std::vector<SeedArgs> seed(n); std::vector<CubArgs> cub(n); std::vector<XyArgs> xy(n);
    std::vector<WtaArgs> wta(n); std::vector<PrepArgs> prep(n); std::vector<ColsumArgs> cs(4 * n);
    std::vector<DsumArgs> dsum(n); std::vector<CtlArgs> ctl(n); std::vector<FrameArgs> frame(n);
    std::vector<Outs> outs(n);
    std::vector<GatherArgs> gather(n);
    std::vector<WnetArgs> wnet(n);
    std::vector<LinArgs> lin(n);
    b->max_lin_blocks = 0;
    b->max_gather = 0;
    b->max_wn_H1 = b->max_wn_n = 0;
    b->max_elems = b->max_cub = b->max_K = b->max_ld = b->max_ent = 0;
    b->max_splits = 1;
    for (int i = 0; i < n; ++i) {
        dae_decoder* d = ds[i];
        const dae_mesh* m = ms[i];
        Workspace& w = d->ws;
        const int r = d->r, L = d->L, N = d->N;
        const int np = d->np, nsys = np + r;   // linear subspace size, system size
        const int ob = out_bf16_of(d->prec);
        const int ld0 = (int)round_up(r, kKPad);
        seed[i] = SeedArgs{w.ns, w.qbar + np, w.qbar_dot + np, dt, h, r, w.Cp, ld0, w.X[0], w.Xh[0],
                           w.Xl[0], d->prec == DAE_TF32 ? kStoreTF32 : ob, w.zvec, np};
        b->max_elems = std::max(b->max_elems, w.Cp * ld0);
        Outs& o = outs[i];
        const bool gout = gram_out(d, m);
        o.u = w.u; o.J = w.J + (size_t)np * N; o.dJ = w.dJ; o.HDD = w.HDD;
        o.row_part = w.row_part; o.row_stride = w.row_stride;
        o.mdof = m->mdof; o.f_ext = hasf[i] ? w.f_ext : nullptr; o.a_out = w.a;
        if (gout) {
            o.gram = true;
            o.n_map = 12 * ncub[i];
            o.pext = hasf[i] ? w.pext : nullptr;
            gather[i] = gs_gather_args(d, m, ncub[i]);
            b->max_gather = std::max(b->max_gather, gather[i].n_rows);
        } else {
            memset(&gather[i], 0, sizeof(GatherArgs));
        }
        CubArgs& ca = cub[i];
        memset(&ca, 0, sizeof ca);
        ca.w_stride = ncub[i];
        ca.u = w.u; ca.J = w.J; ca.N = N; ca.r = nsys; ca.X = m->X; ca.tets = m->tets; ca.Bm = m->Bm;
        ca.np = np; ca.pv = np > 0 ? w.zpv + np : nullptr;
        ca.vol = m->vol; ca.n_tet = m->n_tet; ca.material = m->material; ca.mu = (float)m->mu;
        ca.lam = (float)m->lam; ca.cub_tets = w.cub_tets; ca.cub_w = pred[i] ? w.wn_w : w.cub_w;
        ca.n_cub = ncub[i];
        memset(&wnet[i], 0, sizeof(WnetArgs));
        if (pred[i]) {
            // cubature weights from the system's weight network at its first evaluation
            wnet[i] = wnet_args(d, w.cub_tets, ncub[i], w.wn_w, w.ns, 1);
            b->max_wn_H1 = std::max(b->max_wn_H1, w.wn_H1);
            b->max_wn_n = std::max(b->max_wn_n, ncub[i]);
        }
        ca.fe_w = w.fe_w; ca.fe_dof = w.fe_dof; ca.part = w.cub_part; ca.energy = w.cub_energy;
        ca.stride = w.cub_stride; ca.ns = w.ns; ca.eval_flag = w.eval_flag;
        ca.Jc = gout ? w.Jc : nullptr; ca.ldc = w.Rt * 128;
        ca.n_parts = cubature_parts(ncub[i], ctx->sm_count);
        b->max_cub = std::max(b->max_cub, ca.n_parts);
        const Layer& top = d->layers[L - 1];
        const int K = top.n_in;
        const int kb = (K + 1023) / 1024;
        const bool gram = w.G && w.G_mesh == m->id;
        WtaArgs& wa = wta[i];
        memset(&wa, 0, sizeof wa);
        wa.fe_w = w.fe_w; wa.fe_dof = w.fe_dof; wa.dt2 = dt * dt;
        // coupled: the tie forces of the domain's tie vertices follow the cubature pairs
        wa.n_pairs = 12 * ncub[i] + (cpl ? 3 * cpl->ntv_dom[i] : 0);
        wa.Wp = top.W; wa.ldp = top.ld; wa.K = K;
        memset(&xy[i], 0, sizeof xy[i]);
        if (gout) {
            wa.W = nullptr; wa.N = 0; wa.gy = w.gy;
            wa.pext = hasf[i] ? w.pext : nullptr;
            wa.pext_scale = (float)(-dt * dt);
        } else if (gram) {
            wa.W = w.G; wa.ld = w.ldG; wa.N = K; wa.a = w.xy;
            wa.pext = hasf[i] ? w.pext : nullptr;
            wa.pext_scale = (float)(-dt * dt);
            xy[i] = XyArgs{w.X[(L - 1) & 1], top.ld, K, r, w.zvec, h, w.xy, w.ns};
        } else {
            wa.W = top.W; wa.ld = top.ld; wa.N = N; wa.a = w.a;
        }
        wa.nsplit_dense = std::max(1, std::min(128, std::min((wa.N + 63) / 64, (4 * ctx->sm_count + kb - 1) / kb)));
        wa.nsplit_pairs = std::max(1, std::min(kMaxPairSplits, (wa.n_pairs + 15) / 16));
        wa.part = w.bwd_part[0]; wa.ns = w.ns;
        if (gout) wa.nsplit_dense = 0;
        int in_split = wa.nsplit_dense + wa.nsplit_pairs + (wa.pext ? 1 : 0) + (wa.gy ? 1 : 0);
        memset(&lin[i], 0, sizeof(LinArgs));
        if (np > 0) {
            LinArgs& la = lin[i];
            la.X = w.X[(L - 1) & 1]; la.K = K; la.ldx = top.ld; la.r = r; la.np = np;
            la.V = w.V; la.part = w.lin_part; la.vz = w.bwd_part[0] + (size_t)in_split * K;
            la.zpv = w.zpv; la.ns = w.ns; la.q_in = nullptr; la.qbar = w.qbar;
            la.qbar_dot = w.qbar_dot; la.dt = dt;
            b->max_lin_blocks = std::max(b->max_lin_blocks, w.lin_blocks);
            in_split += 1;
        }
        b->max_K = std::max(b->max_K, K);
        b->max_splits = std::max(b->max_splits, in_split);
        PrepArgs& pa = prep[i];
        memset(&pa, 0, sizeof pa);
        pa.a.n_o = d->widths[L - 1]; pa.a.r = r;
        pa.a.in_part = w.bwd_part[0]; pa.a.in_split = in_split; pa.a.in_ncol = 1;
        pa.a.S1 = w.S1[L - 2]; pa.a.T = w.T[L - 2]; pa.a.ns = w.ns;
        pa.Cb = w.Cb; pa.ld = d->layers[L - 2].ldT;
        pa.g32 = w.G32[0]; pa.gh = w.Gh[0]; pa.gl = w.Gl[0];
        pa.out_f32 = (d->prec == DAE_TF32) ? 2 : 0; pa.out_bf16 = ob;
        b->max_ld = std::max(b->max_ld, pa.ld);
        AsmArgs aa;
        memset(&aa, 0, sizeof aa);
        aa.r = nsys; aa.dt = dt; aa.h = h;
        aa.rq = r; aa.np = np; aa.lin_part = w.lin_part; aa.lin_blocks = w.lin_blocks;
        aa.UMU = w.UMU; aa.Uf = hasf[i] ? w.Uf : nullptr; aa.qbar = w.qbar; aa.qbar_dot = w.qbar_dot;
        aa.row_part = w.row_part; aa.n_row_blocks = gout ? w.Gt : w.n_row_blocks;
        aa.row_stride = w.row_stride;
        aa.cub_part = w.cub_part; aa.cub_energy = w.cub_energy; aa.n_cub = ncub[i];
        aa.cub_stride = w.cub_stride; aa.cub_parts = ca.n_parts;
        aa.bwd_part = w.bwd_part[1]; aa.bwd_split = 1;
        aa.red = w.red; aa.ns = w.ns; aa.control = cpl ? 0 : 1;
        aa.tol = opts.tol; aa.c_armijo = opts.c_armijo; aa.max_iter = opts.max_iter;
        aa.max_step = opts.max_step; aa.xtol = opts.xtol;
        aa.max_halvings = opts.max_halvings; aa.max_evals = opts.max_evals;
        aa.eval_flag = w.eval_flag; aa.status = ctx->d_status;
        aa.lu = cpl ? nullptr : w.lu;
        if (cpl) {
            // coupled: each domain's phi and A only; the global decision reads the flags
            aa.eval_flag = nullptr;
            aa.status = nullptr;
            const Layer& tl = d->layers[L - 1];
            tdom[i] = TieDom{w.X[(L - 1) & 1], tl.ld, tl.W, tl.ld, tl.b, tl.n_in, r, cpl->off[i], w.ns,
                             w.red, w.fe_w, w.fe_dof, 12 * ncub[i], w.eval_flag};
        }
        assemble_parts(aa, &cs[4 * i], dsum[i], ctl[i]);
        for (int k = 0; k < 4; ++k) b->max_ent = std::max(b->max_ent, cs[4 * i + k].n_ent);
    }
    std::vector<ChainJob> jobs;
    std::vector<int> stage_off;
    TRY(batch_chain_jobs(ctx, ds, true, outs, dt, h, jobs, stage_off, b->fwd));
    TRY(batch_chain_jobs(ctx, ds, false, outs, dt, h, jobs, stage_off, b->rev));
    // one device allocation for everything the graph reads
    size_t off = 0;
    auto place = [&](size_t bytes) { size_t o = off; off += round_up(bytes, 256); return o; };
    const size_t o_seed = place(n * sizeof(SeedArgs)), o_cub = place(n * sizeof(CubArgs));
    const size_t o_xy = place(n * sizeof(XyArgs)), o_wta = place(n * sizeof(WtaArgs));
    const size_t o_prep = place(n * sizeof(PrepArgs)), o_cs = place(4 * n * sizeof(ColsumArgs));
    const size_t o_ds = place(n * sizeof(DsumArgs)), o_ctl = place(n * sizeof(CtlArgs));
    const size_t o_lin = place(n * sizeof(LinArgs));
    const size_t o_fr = place(n * sizeof(FrameArgs));
    const size_t o_ga = place(n * sizeof(GatherArgs));
    const size_t o_wn = place(n * sizeof(WnetArgs));
    const size_t o_q0 = place((size_t)n * kMaxR * sizeof(double));
    const size_t o_qo = place((size_t)n * kMaxR * sizeof(double));
    const size_t o_ns = place((size_t)n * sizeof(NewtonState));
    const size_t o_jobs = place(jobs.size() * sizeof(ChainJob));
    const size_t o_st = place(stage_off.size() * sizeof(int));
    const size_t o_gb = place(sizeof(GridBar));
    const size_t o_fl = place(sizeof(int));
    CU(ctx, cudaMalloc(&b->dev, off));
    char* D = b->dev;
    b->seed = (SeedArgs*)(D + o_seed); b->cub = (CubArgs*)(D + o_cub); b->xy = (XyArgs*)(D + o_xy);
    b->wta = (WtaArgs*)(D + o_wta); b->prep = (PrepArgs*)(D + o_prep); b->cs = (ColsumArgs*)(D + o_cs);
    b->ds = (DsumArgs*)(D + o_ds); b->ctl = (CtlArgs*)(D + o_ctl); b->frame = (FrameArgs*)(D + o_fr);
    b->lin = (LinArgs*)(D + o_lin);
    b->gather = (GatherArgs*)(D + o_ga);
    b->wnet = (WnetArgs*)(D + o_wn);
    b->q0 = (double*)(D + o_q0); b->qout = (double*)(D + o_qo); b->ns_out = (NewtonState*)(D + o_ns);
    b->jobs = (ChainJob*)(D + o_jobs); b->stage_off = (int*)(D + o_st); b->gb = (GridBar*)(D + o_gb);
    b->flag = (int*)(D + o_fl);
    for (int i = 0; i < n; ++i)
        frame[i] = FrameArgs{ds[i]->ws.ns, b->q0 + (size_t)i * kMaxR, b->qout + (size_t)i * kMaxR,
                             ds[i]->np + ds[i]->r};
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    CU(ctx, up(b->seed, seed.data(), n * sizeof(SeedArgs)));
    CU(ctx, up(b->cub, cub.data(), n * sizeof(CubArgs)));
    CU(ctx, up(b->xy, xy.data(), n * sizeof(XyArgs)));
    CU(ctx, up(b->wta, wta.data(), n * sizeof(WtaArgs)));
    CU(ctx, up(b->prep, prep.data(), n * sizeof(PrepArgs)));
    CU(ctx, up(b->cs, cs.data(), 4 * n * sizeof(ColsumArgs)));
    CU(ctx, up(b->lin, lin.data(), n * sizeof(LinArgs)));
    CU(ctx, up(b->ds, dsum.data(), n * sizeof(DsumArgs)));
    CU(ctx, up(b->ctl, ctl.data(), n * sizeof(CtlArgs)));
    CU(ctx, up(b->frame, frame.data(), n * sizeof(FrameArgs)));
    CU(ctx, up(b->gather, gather.data(), n * sizeof(GatherArgs)));
    CU(ctx, up(b->wnet, wnet.data(), n * sizeof(WnetArgs)));
    CU(ctx, up(b->jobs, jobs.data(), jobs.size() * sizeof(ChainJob)));
    if (cpl) TRY(upload_coupling(ctx, *cpl, tdom, dt, h, opts));
    CU(ctx, up(b->stage_off, stage_off.data(), stage_off.size() * sizeof(int)));
    CU(ctx, cudaMemset(b->gb, 0, sizeof(GridBar)));
    b->epoch = ctx->timeout_epoch;

    // graph: begin -> WHILE(any system running) { evaluation of all systems } -> end
    if (!ctx->cap_stream) CU(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t s = ctx->cap_stream;
    const dae_prec prec = ds[0]->prec;
    b->n = n;
    cudaGraph_t g = nullptr;
    CU(ctx, cudaGraphCreate(&g, 0));
    dae_status st = DAE_OK;
    const cudaStream_t saved_stream = ctx->stream;
    const unsigned saved_prof = ctx->prof_on;
    const long long saved_launches = ctx->launches;
    ctx->stream = s;
    ctx->prof_on = 0;
    do {
        cudaGraphConditionalHandle hc;
        if (cudaGraphConditionalHandleCreate(&hc, g, 0, 0) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        if (cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        launch_frame_begin_batched(s, b->frame, n, hc, 1);
        if (cpl) launch_coupled_begin(s, cpl->args);
        if (cudaStreamEndCapture(s, &g) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        cudaGraphNode_t a, loop;
        cudaGraph_t body;
        if ((st = sole_sink(ctx, g, &a))) break;
        if ((st = add_while(ctx, g, &a, hc, &loop, &body))) break;
        if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        const dae_status es = enqueue_batch_eval(ctx, b, prec, hc, nullptr);
        cudaGraph_t body2 = body;
        const cudaError_t ce = cudaStreamEndCapture(s, &body2);
        if (es) { st = es; break; }
        if (ce != cudaSuccess) { st = fail(ctx, DAE_ERR_CUDA, "capture failed: %s", cudaGetErrorString(ce)); break; }
        if (cudaStreamBeginCaptureToGraph(s, g, &loop, nullptr, 1, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        launch_frame_end_batched(s, b->frame, n);
        if (cudaStreamEndCapture(s, &g) != cudaSuccess) { st = DAE_ERR_CUDA; break; }
        const cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
        if (ie != cudaSuccess) { st = fail(ctx, DAE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie)); break; }
    } while (0);
    ctx->stream = saved_stream;
    ctx->prof_on = saved_prof;
    ctx->launches = saved_launches;
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (st) {
        if (ctx->err.empty()) fail(ctx, st, "batch graph construction failed");
        b->gexec = nullptr;
        b->key.clear();
        return st;
    }
    return DAE_OK;
}

}  // namespace

// =============================================================== C ABI ====
// The forward pass in exact multicomplex columns (CUDA-core FP32 kernels): the seed
// and every layer with the exact epilogue, into the outputs of o (u, J, Hqq, dJ).
dae_status enqueue_forward_exact(dae_decoder* d, const double* dq, double dt, double h, int mode,
                                 const Outs& o) {
    dae_ctx* ctx = d->ctx;
    Workspace& w = d->ws;
    cudaStream_t s = ctx->stream;
    const int r = d->r, L = d->L;
    const int Cpx = pad_cols_exact(r);
    if (!w.Xe[0] || w.Cpx != Cpx) {
        CU(ctx, cudaStreamSynchronize(s));
        dfree(w.Xe[0]); dfree(w.Xe[1]);
        TRY(dmalloc(ctx, &w.Xe[0], (size_t)Cpx * w.ldx_max));
        TRY(dmalloc(ctx, &w.Xe[1], (size_t)Cpx * w.ldx_max));
        w.Cpx = Cpx;
    }
    const int ld0 = (int)round_up(r, kKPad);
    {
        Phase p(ctx, DAE_PHASE_SEED, 1);
        launch_seed_exact(s, dq, w.qbar, w.qbar_dot, dt, h, mode, r, Cpx, ld0, w.Xe[0]);
    }
    for (int l = 0; l < L; ++l) {
        FwdArgs a;
        fill_fwd_args(d, l, a);
        a.Cp = Cpx;
        a.exact = 1;
        a.X = w.Xe[l & 1]; a.Xh = a.Xl = nullptr;
        a.Y = a.last ? nullptr : w.Xe[(l + 1) & 1];
        a.Yh = a.Yl = nullptr; a.out_bf16 = 0; a.out_f32 = 1;
        a.S1 = nullptr; a.T = nullptr;
        a.inv_h = 1.0 / h; a.inv_h2 = 1.0 / (h * h); a.inv_h3 = 1.0 / (h * h * h);
        a.inv_dt2 = 1.0 / (dt * dt);
        if (a.last) { a.u = o.u; a.J = o.J; a.dJ = o.dJ; a.HDD = o.HDD; a.Hqq = o.Hqq; }
        Phase p(ctx, a.last ? DAE_PHASE_FWD_OUT : DAE_PHASE_FWD_HIDDEN, 1);
        launch_fwd_simt(s, a);
    }
    CU(ctx, cudaGetLastError());
    return DAE_OK;
}

extern "C" {

int dae_version(void) { return DAE_VERSION; }

const char* dae_status_string(dae_status s) {
    switch (s) {
        case DAE_OK: return "DAE_OK";
        case DAE_ERR_INVALID_ARG: return "DAE_ERR_INVALID_ARG";
        case DAE_ERR_CUDA: return "DAE_ERR_CUDA";
        case DAE_ERR_OOM: return "DAE_ERR_OOM";
        case DAE_ERR_NOT_CONVERGED: return "DAE_ERR_NOT_CONVERGED";
        case DAE_ERR_NONFINITE: return "DAE_ERR_NONFINITE";
        case DAE_ERR_SINGULAR: return "DAE_ERR_SINGULAR";
        case DAE_ERR_INVERTED: return "DAE_ERR_INVERTED";
        case DAE_ERR_TIMEOUT: return "DAE_ERR_TIMEOUT";
        case DAE_ERR_UNSUPPORTED: return "DAE_ERR_UNSUPPORTED";
    }
    return "unknown";
}

void dae_default_newton_opts(dae_newton_opts* o) {
    if (!o) return;
    o->max_iter = 5;
    o->max_evals = 8;
    o->max_halvings = 8;
    o->tol = 1e-8;
    o->c_armijo = 1e-4;
    o->h_cs = std::ldexp(1.0, -20);
    o->max_step = 0.5;
    o->xtol = 1e-6;
}

dae_status dae_create(dae_ctx** out, int device, void* stream) {
    if (!out) return DAE_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DAE_ERR_CUDA;
    }
    dae_ctx* ctx = new dae_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return DAE_ERR_CUDA; }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess) { delete ctx; return DAE_ERR_OOM; }
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
    if (cudaMalloc(&ctx->d_kcount, sizeof(unsigned long long)) != cudaSuccess) { delete ctx; return DAE_ERR_OOM; }
    cudaMemsetAsync(ctx->d_kcount, 0, sizeof(unsigned long long), ctx->stream);
    *out = ctx;
    return DAE_OK;
}

dae_status dae_destroy(dae_ctx* ctx) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx->d_status);
    dfree(ctx->d_kcount);
    dfree(ctx->dstage);
    free_batch(ctx);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cublas) cublasDestroy((cublasHandle_t)ctx->cublas);
    for (auto& rec : ctx->recs) { cudaEventDestroy(rec.a); cudaEventDestroy(rec.b); }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return DAE_OK;
}

const char* dae_last_error(const dae_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dae_status dae_sync(dae_ctx* ctx) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    CU(ctx, cudaSetDevice(ctx->device));
    return check_device_status(ctx);
}

dae_status dae_load_decoder(dae_ctx* ctx, int n_layers, const int* widths, const float* const* W,
                            const float* const* b, dae_act act, dae_prec prec, dae_decoder** out) {
    if (!ctx || !out) return DAE_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_layers < 2 || !widths || !W || !b)
        return fail(ctx, DAE_ERR_INVALID_ARG, "need >= 2 layers and widths/W/b arrays");
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] <= 0) return fail(ctx, DAE_ERR_INVALID_ARG, "width %d is %d", l, widths[l]);
    if (widths[0] > kMaxR) return fail(ctx, DAE_ERR_UNSUPPORTED, "latent size %d > %d", widths[0], kMaxR);
    if (act < DAE_ACT_TANH || act > DAE_ACT_LINEAR) return fail(ctx, DAE_ERR_INVALID_ARG, "bad activation");
    if (prec < DAE_FP32 || prec > DAE_BF16X3) return fail(ctx, DAE_ERR_INVALID_ARG, "bad precision");
    CU(ctx, cudaSetDevice(ctx->device));
    dae_decoder* d = new dae_decoder();
    d->ctx = ctx;
    d->L = n_layers;
    d->r = widths[0];
    d->N = widths[n_layers];
    d->widths.assign(widths, widths + n_layers + 1);
    d->act = act;
    d->prec = DAE_FP32;
    d->layers.resize(n_layers);
    auto cleanup = [&](dae_status st) {
        dae_free_decoder(d);
        return st;
    };
    for (int l = 0; l < n_layers; ++l) {
        Layer& ly = d->layers[l];
        ly.n_in = widths[l];
        ly.n_out = widths[l + 1];
        ly.ld = (int)round_up(ly.n_in, kKPad);
        ly.m_pad = (int)round_up(ly.n_out, kRowTile);
        if (!W[l] || !b[l]) return cleanup(fail(ctx, DAE_ERR_INVALID_ARG, "layer %d arrays missing", l));
        dae_status st = dmalloc(ctx, &ly.W, (size_t)ly.m_pad * ly.ld);
        if (st) return cleanup(st);
        st = dmalloc(ctx, &ly.b, (size_t)ly.n_out);
        if (st) return cleanup(st);
        cudaError_t e = cudaMemcpy2DAsync(ly.W, (size_t)ly.ld * sizeof(float), W[l],
                                          (size_t)ly.n_in * sizeof(float), (size_t)ly.n_in * sizeof(float),
                                          ly.n_out, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ly.b, b[l], (size_t)ly.n_out * sizeof(float), cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess)
            return cleanup(fail(ctx, DAE_ERR_CUDA, "weight upload: %s", cudaGetErrorString(e)));
    }
    dae_status st = alloc_workspace(d);
    if (st) return cleanup(st);
    st = dae_decoder_set_precision(d, prec);
    if (st) return cleanup(st);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return cleanup(fail(ctx, DAE_ERR_CUDA, "decoder upload failed"));
    *out = d;
    return DAE_OK;
}

dae_status dae_decoder_set_precision(dae_decoder* d, dae_prec prec) {
    if (!d) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = d->ctx;
    if (prec < DAE_FP32 || prec > DAE_BF16X3) return fail(ctx, DAE_ERR_INVALID_ARG, "bad precision");
    CU(ctx, cudaSetDevice(ctx->device));
    // the cached frame graph bakes the layer chains' job, partial-tile and counter
    // buffers, which build_chains below frees and reallocates: never replay it again
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    drop_graph(d->ws);
    // a chain plan belongs to the precision it was set or tuned for; the exact
    // multicomplex activation to the FP32 form
    d->plan_prec = -1;
    if (prec != DAE_FP32) d->cs_exact = 0;
    d->plan_split[0].clear(); d->plan_split[1].clear();
    d->plan_rep[0].clear(); d->plan_rep[1].clear();
    if (prec == DAE_BF16 || prec == DAE_BF16X3) {
        for (auto& ly : d->layers) {
            size_t n = (size_t)ly.m_pad * ly.ld;
            if (!ly.Wh) TRY(dmalloc(ctx, &ly.Wh, n));
            if (prec == DAE_BF16X3 && !ly.Wl) TRY(dmalloc(ctx, &ly.Wl, n));
            launch_split_bf16(ctx->stream, ly.W, ly.Wh, prec == DAE_BF16X3 ? ly.Wl : nullptr, n);
        }
    }
    if (prec == DAE_TF32) {
        for (auto& ly : d->layers) {
            size_t n = (size_t)ly.m_pad * ly.ld;
            if (!ly.Wr) TRY(dmalloc(ctx, &ly.Wr, n));
            launch_round_tf32(ctx->stream, ly.W, ly.Wr, n);
        }
    }
    CU(ctx, cudaGetLastError());
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (prec != DAE_FP32) {
        // TMA descriptors of every layer: A = weights [m_pad][ld], B = input activations [Cp][ld]
        const bool f32 = (prec == DAE_TF32);
        for (int l = 0; l < d->L; ++l) {
            Layer& ly = d->layers[l];
            const int buf = l & 1;
            bool ok = make_tmap(&ly.tm[0], f32 ? (const void*)ly.Wr : (const void*)ly.Wh, f32, ly.ld,
                                ly.m_pad, 128);
            ok = ok && make_tmap(&ly.tm[2], f32 ? (const void*)d->ws.X[buf] : (const void*)d->ws.Xh[buf],
                                 f32, ly.ld, d->ws.Cp, d->ws.Cp);
            if (prec == DAE_BF16X3) {
                ok = ok && make_tmap(&ly.tm[1], ly.Wl, false, ly.ld, ly.m_pad, 128);
                ok = ok && make_tmap(&ly.tm[3], d->ws.Xl[buf], false, ly.ld, d->ws.Cp, d->ws.Cp);
            } else {
                ly.tm[1] = ly.tm[0];
                ly.tm[3] = ly.tm[2];
            }
            ly.tm_ok = ok;
            if (!ok) return fail(ctx, DAE_ERR_UNSUPPORTED, "tensor map encoding failed for layer %d", l);
        }
        // reverse pass: W_l^T (K-major, K = n_out) for every hidden layer, and its B operand
        // g_l (ping-pong buffer (L-2-l) & 1)
        for (int l = 0; l < d->L - 1; ++l) {
            Layer& ly = d->layers[l];
            ly.ldT = (int)round_up(ly.n_out, kKPad);
            ly.mT_pad = (int)round_up(ly.n_in, kRowTile);
            const size_t nt = (size_t)ly.mT_pad * ly.ldT;
            if (!ly.WT) {
                TRY(dmalloc(ctx, &ly.WT, nt));
                launch_transpose(ctx->stream, ly.W, ly.ld, ly.n_out, ly.n_in, ly.WT, ly.ldT);
            }
            if (prec == DAE_TF32) {
                if (!ly.WTr) TRY(dmalloc(ctx, &ly.WTr, nt));
                launch_round_tf32(ctx->stream, ly.WT, ly.WTr, nt);
            } else {
                if (!ly.WTh) TRY(dmalloc(ctx, &ly.WTh, nt));
                if (prec == DAE_BF16X3 && !ly.WTl) TRY(dmalloc(ctx, &ly.WTl, nt));
                launch_split_bf16(ctx->stream, ly.WT, ly.WTh, prec == DAE_BF16X3 ? ly.WTl : nullptr, nt);
            }
            const int gb = (d->L - 2 - l) & 1;
            bool ok = make_tmap(&ly.tmR[0], f32 ? (const void*)ly.WTr : (const void*)ly.WTh, f32, ly.ldT,
                                ly.mT_pad, 128);
            ok = ok && make_tmap(&ly.tmR[2], f32 ? (const void*)d->ws.G32[gb] : (const void*)d->ws.Gh[gb],
                                 f32, ly.ldT, d->ws.Cb, d->ws.Cb);
            if (prec == DAE_BF16X3) {
                ok = ok && make_tmap(&ly.tmR[1], ly.WTl, false, ly.ldT, ly.mT_pad, 128);
                ok = ok && make_tmap(&ly.tmR[3], d->ws.Gl[gb], false, ly.ldT, d->ws.Cb, d->ws.Cb);
            } else {
                ly.tmR[1] = ly.tmR[0];
                ly.tmR[3] = ly.tmR[2];
            }
            ly.tmR_ok = ok;
            if (!ok) return fail(ctx, DAE_ERR_UNSUPPORTED, "reverse tensor map failed for layer %d", l);
        }
        CU(ctx, cudaGetLastError());
        CU(ctx, cudaStreamSynchronize(ctx->stream));
    }
    d->prec = prec;
    d->id = g_dec_ids++;   // cached grouped plans of the old form no longer match
    d->ws.chain_ok = false;
    if (prec != DAE_FP32) TRY(build_chains(d));
    d->prec = prec;
    return DAE_OK;
}

dae_status dae_decoder_get_chain_plan(const dae_decoder* d, int dir, int* split, int* rep) {
    if (!d || (dir != 0 && dir != 1) || !split || !rep) return DAE_ERR_INVALID_ARG;
    if (d->prec == DAE_FP32 || !d->ws.chain_ok)
        return fail(d->ctx, DAE_ERR_UNSUPPORTED, "the layer chains run in the tensor-core precisions only");
    std::vector<ChainJob> fj, rj;
    size_t part, cf, cr;
    chain_jobs(d, fj, rj, part, cf, cr);
    for (int l = 0; l < d->L - 1; ++l) {
        const ChainJob& j = dir == 0 ? fj[l] : rj[d->L - 2 - l];
        split[l] = j.split;
        rep[l] = j.solo ? 0 : j.rep;
    }
    return DAE_OK;
}

dae_status dae_decoder_set_chain_plan(dae_decoder* d, int dir, const int* split, const int* rep) {
    if (!d || (dir != 0 && dir != 1)) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = d->ctx;
    if (d->prec == DAE_FP32 || !d->ws.chain_ok)
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the layer chains run in the tensor-core precisions only");
    CU(ctx, cudaSetDevice(ctx->device));
    const int n = d->L - 1;
    std::vector<int> sp(n), rp(n);
    if (split && rep) {
        TRY(check_plan(d, dir, split, rep));
        sp.assign(split, split + n);
        rp.assign(rep, rep + n);
    } else {
        // NULL arrays: back to the fixed heuristic for this direction
        std::vector<ChainJob> fj, rj;
        size_t part, cf, cr;
        const int saved = d->plan_prec;
        d->plan_prec = -1;
        chain_jobs(d, fj, rj, part, cf, cr);
        d->plan_prec = saved;
        for (int l = 0; l < n; ++l) {
            const ChainJob& j = dir == 0 ? fj[l] : rj[n - 1 - l];
            sp[l] = j.split;
            rp[l] = j.rep;
        }
    }
    if (d->plan_prec != (int)d->prec || (int)d->plan_split[1 - dir].size() != n) {
        // the other direction keeps its current plan
        std::vector<int> os(n), orp(n);
        TRY(dae_decoder_get_chain_plan(d, 1 - dir, os.data(), orp.data()));
        d->plan_split[1 - dir] = os;
        d->plan_rep[1 - dir] = orp;
    }
    d->plan_split[dir] = sp;
    d->plan_rep[dir] = rp;
    d->plan_prec = (int)d->prec;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    drop_graph(d->ws);
    d->id = g_dec_ids++;   // cached grouped plans bake the job lists
    return build_chains(d);
}

dae_status dae_decoder_autotune(dae_decoder* d, int reps, double* ms) {
    if (!d) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = d->ctx;
    if (d->prec == DAE_FP32 || !d->ws.chain_ok)
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the layer chains run in the tensor-core precisions only");
    if (reps < 1) reps = 20;
    CU(ctx, cudaSetDevice(ctx->device));
    Workspace& w = d->ws;
    const int L = d->L, n = L - 1, G = ctx->sm_count;
    // room for the largest split any candidate may take
    {
        std::vector<ChainJob> fj, rj;
        size_t part, cf, cr;
        chain_jobs(d, fj, rj, part, cf, cr);
        size_t need = 1;
        for (const auto& j : fj) need = std::max(need, (size_t)j.tiles * 8 * (w.Cp + 1) * 128);
        for (const auto& j : rj) need = std::max(need, (size_t)j.tiles * 8 * (w.Cb + 1) * 128);
        need = std::max(need, (size_t)G * 2 * (w.Cp + 1) * 128);
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(w.chain_part);
        TRY(dmalloc(ctx, &w.chain_part, need));
    }
    double out[4] = {0, 0, 0, 0};
    for (int dir = 0; dir < 2; ++dir) {
        std::vector<ChainJob> fj, rj;
        size_t part, cf, cr;
        chain_jobs(d, fj, rj, part, cf, cr);
        std::vector<ChainJob> jobs = dir == 0 ? fj : rj;   // launch order
        const std::vector<ChainJob> start = jobs;
        double best;
        TRY(time_chain(d, dir, jobs, reps, &best));
        // coordinate descent over the layers, one pass: a candidate replaces the current
        // plan of its layer when it is faster by more than 1 % (timing noise)
        for (int i = 0; i < n; ++i) {
            for (auto c : plan_candidates(jobs[i], G)) {
                if (c.first == jobs[i].split && c.second == (jobs[i].solo ? 0 : jobs[i].rep)) continue;
                std::vector<ChainJob> trial = jobs;
                trial[i].split = c.first;
                trial[i].rep = c.second == 0 ? 1 : c.second;
                trial[i].solo = c.second == 0 ? 1 : 0;
                double t;
                TRY(time_chain(d, dir, trial, reps, &t));
                if (t < 0.99 * best) { best = t; jobs = trial; }
            }
        }
        // runs of consecutive small layers on CTA 0 alone at either end of the chain (a run
        // hands its activations from layer to layer inside CTA 0, with no wait on other
        // CTAs' ready counters between its layers)
        auto solo_ok = [&](const ChainJob& j) {
            for (auto c : plan_candidates(j, G)) if (c.second == 0) return true;
            return false;
        };
        for (int len = 2; len <= n; ++len) {
            for (int end = 0; end < 2; ++end) {
                const int a = end == 0 ? 0 : n - len;
                bool ok = true;
                for (int i = a; i < a + len; ++i) ok = ok && solo_ok(jobs[i]);
                if (!ok) continue;
                std::vector<ChainJob> trial = jobs;
                for (int i = a; i < a + len; ++i) { trial[i].split = 1; trial[i].rep = 1; trial[i].solo = 1; }
                double t;
                TRY(time_chain(d, dir, trial, reps, &t));
                if (t < 0.99 * best) { best = t; jobs = trial; }
            }
        }
        // the start and the result timed again, interleaved
        double t0 = 0, t1 = 0;
        for (int k = 0; k < 3; ++k) {
            double a, b;
            TRY(time_chain(d, dir, start, reps, &a));
            TRY(time_chain(d, dir, jobs, reps, &b));
            t0 += a / 3;
            t1 += b / 3;
        }
        if (t1 > t0) { jobs = start; t1 = t0; }   // never keep a slower plan
        out[2 * dir] = t0;
        out[2 * dir + 1] = t1;
        std::vector<int> sp(n), rp(n);
        for (int i = 0; i < n; ++i) {
            const int l = dir == 0 ? i : n - 1 - i;   // layer order
            sp[l] = jobs[i].split;
            rp[l] = jobs[i].solo ? 0 : jobs[i].rep;
        }
        if (d->plan_prec != (int)d->prec || (int)d->plan_split[1 - dir].size() != n) {
            std::vector<int> os(n), orp(n);
            TRY(dae_decoder_get_chain_plan(d, 1 - dir, os.data(), orp.data()));
            d->plan_split[1 - dir] = os;
            d->plan_rep[1 - dir] = orp;
        }
        d->plan_split[dir] = sp;
        d->plan_rep[dir] = rp;
        d->plan_prec = (int)d->prec;
    }
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    drop_graph(w);
    d->id = g_dec_ids++;
    TRY(build_chains(d));
    if (ms) memcpy(ms, out, sizeof out);
    return DAE_OK;
}

dae_status dae_decoder_attach_wnet(dae_decoder* d, const int* widths, const float* const* W,
                                   const float* const* b) {
    if (!d) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = d->ctx;
    if (!widths || !W || !b) return fail(ctx, DAE_ERR_INVALID_ARG, "widths, W and b required");
    for (int l = 0; l < 4; ++l)
        if (!W[l] || !b[l]) return fail(ctx, DAE_ERR_INVALID_ARG, "weight network layer %d missing", l);
    if (widths[0] != d->N) return fail(ctx, DAE_ERR_INVALID_ARG, "weight network input %d != decoder output %d", widths[0], d->N);
    if (d->np > 0) return fail(ctx, DAE_ERR_UNSUPPORTED, "weight network with a linear subspace");
    for (int l = 1; l <= 3; ++l)
        if (widths[l] <= 0 || widths[l] > kMaxWnetWidth)
            return fail(ctx, DAE_ERR_UNSUPPORTED, "weight network width %d must be in [1, %d]", widths[l], kMaxWnetWidth);
    if (widths[4] <= 0) return fail(ctx, DAE_ERR_INVALID_ARG, "weight network output width %d", widths[4]);
    CU(ctx, cudaSetDevice(ctx->device));
    Workspace& w = d->ws;
    const int N = d->N, H1 = widths[1], H2 = widths[2], H3 = widths[3], T = widths[4];
    const Layer& top = d->layers[d->L - 1];
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    dfree(w.wn_B1); dfree(w.wn_c1); dfree(w.wn_A2); dfree(w.wn_b2); dfree(w.wn_A3); dfree(w.wn_b3);
    dfree(w.wn_A4); dfree(w.wn_b4); dfree(w.wn_h1);
    w.wn_H1 = w.wn_H2 = w.wn_H3 = w.wn_ntet = 0;
    float* A1 = nullptr;
    TRY(dmalloc(ctx, &A1, (size_t)H1 * N));
    auto up = [&](float* dst, const float* src, size_t n) {
        return cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDefault, ctx->stream);
    };
    dae_status st = DAE_OK;
    do {
        if ((st = dmalloc(ctx, &w.wn_B1, (size_t)H1 * top.ld))) break;
        if ((st = dmalloc(ctx, &w.wn_c1, (size_t)H1))) break;
        if ((st = dmalloc(ctx, &w.wn_A2, (size_t)H2 * H1))) break;
        if ((st = dmalloc(ctx, &w.wn_b2, (size_t)H2))) break;
        if ((st = dmalloc(ctx, &w.wn_A3, (size_t)H3 * H2))) break;
        if ((st = dmalloc(ctx, &w.wn_b3, (size_t)H3))) break;
        if ((st = dmalloc(ctx, &w.wn_A4, (size_t)T * H3))) break;
        if ((st = dmalloc(ctx, &w.wn_b4, (size_t)T))) break;
        if ((st = dmalloc(ctx, &w.wn_h1, (size_t)2 * kMaxWnetWidth))) break;   // h1 | h3
        if (up(A1, W[0], (size_t)H1 * N) || up(w.wn_c1, b[0], H1) || up(w.wn_A2, W[1], (size_t)H2 * H1) ||
            up(w.wn_b2, b[1], H2) || up(w.wn_A3, W[2], (size_t)H3 * H2) || up(w.wn_b3, b[2], H3) ||
            up(w.wn_A4, W[3], (size_t)T * H3) || up(w.wn_b4, b[3], T)) {
            st = fail(ctx, DAE_ERR_CUDA, "weight network upload failed");
            break;
        }
        if (!ctx->cublas) {
            cublasHandle_t hnd;
            if (cublasCreate(&hnd) != CUBLAS_STATUS_SUCCESS) { st = fail(ctx, DAE_ERR_CUDA, "cublasCreate failed"); break; }
            ctx->cublas = hnd;
        }
        cublasHandle_t hnd = (cublasHandle_t)ctx->cublas;
        cublasSetStream(hnd, ctx->stream);
        cublasSetMathMode(hnd, CUBLAS_DEFAULT_MATH);
        // B1 = A1 W_L ([H1][ld], row-major) and c1 = A1 b_L + b1: the first layer composed
        // with the decoder's linear output layer (column-major view: B1^T = W_L^T A1^T)
        const float one = 1.f, zero = 0.f;
        cublasStatus_t cs = cublasSgemm(hnd, CUBLAS_OP_N, CUBLAS_OP_N, top.ld, H1, N, &one, top.W, top.ld,
                                        A1, N, &zero, w.wn_B1, top.ld);
        if (cs == CUBLAS_STATUS_SUCCESS)
            cs = cublasSgemv(hnd, CUBLAS_OP_T, N, H1, &one, A1, N, top.b, 1, &one, w.wn_c1, 1);
        if (cs != CUBLAS_STATUS_SUCCESS) { st = fail(ctx, DAE_ERR_CUDA, "weight network composition failed (%d)", (int)cs); break; }
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { st = fail(ctx, DAE_ERR_CUDA, "weight network set-up failed"); break; }
    } while (0);
    dfree(A1);
    if (st) return st;
    w.wn_H1 = H1; w.wn_H2 = H2; w.wn_H3 = H3; w.wn_ntet = T;
    w.graph_ok = false;
    return DAE_OK;
}

dae_status dae_decoder_attach_linear(dae_decoder* d, int np, const float* U) {
    if (!d) return DAE_ERR_INVALID_ARG;
    dae_ctx* ctx = d->ctx;
    if (!U || np < 1) return fail(ctx, DAE_ERR_INVALID_ARG, "U and np >= 1 required");
    if (d->np > 0) return fail(ctx, DAE_ERR_INVALID_ARG, "a linear subspace is already attached");
    if (np + d->r > kMaxR) return fail(ctx, DAE_ERR_UNSUPPORTED, "np + r = %d > %d", np + d->r, kMaxR);
    if (d->prec == DAE_FP32 || !d->ws.chain_ok)
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the linear subspace needs a tensor-core precision");
    if (d->ws.wn_B1) return fail(ctx, DAE_ERR_UNSUPPORTED, "weight network with a linear subspace");
    CU(ctx, cudaSetDevice(ctx->device));
    Workspace& w = d->ws;
    Layer& top = d->layers[d->L - 1];
    const int N = d->N, r = d->r, n = np + r, K = top.n_in;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    float* Ud = nullptr;
    float* T = nullptr;
    TRY(dmalloc(ctx, &Ud, (size_t)np * N));
    TRY(dmalloc(ctx, &T, (size_t)np * top.ld + np));
    CU(ctx, cudaMemcpyAsync(Ud, U, (size_t)np * N * sizeof(float), cudaMemcpyDefault, ctx->stream));
    if (!ctx->cublas) {
        cublasHandle_t hnd;
        if (cublasCreate(&hnd) != CUBLAS_STATUS_SUCCESS) return fail(ctx, DAE_ERR_CUDA, "cublasCreate failed");
        ctx->cublas = hnd;
    }
    cublasHandle_t hnd = (cublasHandle_t)ctx->cublas;
    cublasSetStream(hnd, ctx->stream);
    cublasSetMathMode(hnd, CUBLAS_DEFAULT_MATH);
    // the filtering layer folded into the output layer: W_L <- (I - U U^T) W_L,
    // b_L <- (I - U U^T) b_L (column-major views: W_L is ld x N, U is N x np)
    const float one = 1.f, zero = 0.f, mone = -1.f;
    float* tb = T + (size_t)np * top.ld;
    cublasStatus_t cs = cublasSgemm(hnd, CUBLAS_OP_N, CUBLAS_OP_N, top.ld, np, N, &one, top.W, top.ld,
                                    Ud, N, &zero, T, top.ld);
    if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasSgemm(hnd, CUBLAS_OP_N, CUBLAS_OP_T, top.ld, N, np, &mone, T, top.ld, Ud, N, &one,
                         top.W, top.ld);
    if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasSgemv(hnd, CUBLAS_OP_T, N, np, &one, Ud, N, top.b, 1, &zero, tb, 1);
    if (cs == CUBLAS_STATUS_SUCCESS)
        cs = cublasSgemv(hnd, CUBLAS_OP_N, N, np, &mone, Ud, N, tb, 1, &one, top.b, 1);
    if (cs != CUBLAS_STATUS_SUCCESS) {
        dfree(Ud); dfree(T);
        return fail(ctx, DAE_ERR_CUDA, "filtering layer failed (%d)", (int)cs);
    }
    // system-size buffers: J holds U in its first np rows
    float* J2 = nullptr;
    dae_status st = dmalloc(ctx, &J2, (size_t)n * N);
    if (!st) {
        CU(ctx, cudaMemcpyAsync(J2, Ud, (size_t)np * N * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
        CU(ctx, cudaStreamSynchronize(ctx->stream));
    }
    dfree(Ud); dfree(T);
    if (st) return st;
    dfree(w.J); w.J = J2;
    dfree(w.red); dfree(w.qbar); dfree(w.qbar_dot); dfree(w.q0); dfree(w.qout);
    TRY(dmalloc(ctx, &w.red, red_size(n)));
    TRY(dmalloc(ctx, &w.qbar, (size_t)n));
    TRY(dmalloc(ctx, &w.qbar_dot, (size_t)n));
    TRY(dmalloc(ctx, &w.q0, (size_t)n));
    if (w.rc) TRY(dmalloc(ctx, &w.qout, (size_t)n));
    dfree(w.hist); dfree(w.traj); w.hist_cap = 0;
    dfree(w.fe_w); dfree(w.fe_dof); dfree(w.cub_part); dfree(w.cub_energy); dfree(w.cub_tets);
    w.cub_cap = 0;
    w.lin_blocks = (K + 63) / 64;
    TRY(dmalloc(ctx, &w.V, (size_t)top.ld * np));
    TRY(dmalloc(ctx, &w.UMU, (size_t)np * np));
    TRY(dmalloc(ctx, &w.Uf, (size_t)np));
    TRY(dmalloc(ctx, &w.zpv, (size_t)2 * np));
    TRY(dmalloc(ctx, &w.lin_part, (size_t)w.lin_blocks * np * (1 + 2 * r)));
    if (w.cub_rows)   // the stacked operand's cubature rows hold unfiltered W_L rows
        CU(ctx, cudaMemsetAsync(w.cub_rows, 0xff, (size_t)w.gs_rows_cap * sizeof(int), ctx->stream));
    d->np = np;
    w.V_mesh = 0; w.G_mesh = 0; w.gs_G_mesh = 0; w.pext_valid = false; w.graph_ok = false;
    // operand forms of the filtered output layer (splits / rounding, tensor maps, chains)
    return dae_decoder_set_precision(d, d->prec);
}

dae_status dae_predict_weights(dae_ctx* ctx, const dae_decoder* dec_c, const double* q, int n,
                               const int* tet_ids, float* w_out) {
    TRY(check_common(ctx, dec_c, nullptr));
    dae_decoder* d = const_cast<dae_decoder*>(dec_c);
    if (!d->ws.wn_B1) return fail(ctx, DAE_ERR_INVALID_ARG, "no weight network attached");
    if (!q || n < 0 || (n > 0 && (!tet_ids || !w_out))) return fail(ctx, DAE_ERR_INVALID_ARG, "q, tet_ids, w required");
    if (n > 0 && !on_device(tet_ids))
        for (int i = 0; i < n; ++i)
            if (tet_ids[i] < 0 || tet_ids[i] >= d->ws.wn_ntet)
                return fail(ctx, DAE_ERR_INVALID_ARG, "element %d out of range", tet_ids[i]);
    if (n == 0) return DAE_OK;
    const int r = d->r;
    Stage st(ctx);
    st.need(q, r * 8); st.need(tet_ids, (size_t)n * 4); st.need(w_out, (size_t)n * 4);
    TRY(st.reserve(st.plan));
    const double* dq;
    const int* dt;
    float* dw;
    TRY(st.in(q, r, &dq));
    TRY(st.in(tet_ids, n, &dt));
    TRY(st.inout(w_out, n, &dw, false));
    Outs o;   // hidden layers only matter: no outputs
    TRY(enqueue_forward(d, nullptr, dq, 1.0, std::ldexp(1.0, -20), SEED_FULL, o));
    ctx->launches += 3;
    launch_wnet(ctx->stream, wnet_args(d, dt, n, dw, nullptr, 0));
    CU(ctx, cudaGetLastError());
    TRY(st.finish());
    return DAE_OK;
}

dae_status dae_free_decoder(dae_decoder* d) {
    if (!d) return DAE_ERR_INVALID_ARG;
    cudaSetDevice(d->ctx->device);
    cudaStreamSynchronize(d->ctx->stream);
    for (auto& ly : d->layers) {
        dfree(ly.W); dfree(ly.b); dfree(ly.Wh); dfree(ly.Wl); dfree(ly.Wr);
        dfree(ly.WT); dfree(ly.WTh); dfree(ly.WTl); dfree(ly.WTr);
    }
    free_workspace(d->ws);
    delete d;
    return DAE_OK;
}

dae_status dae_load_mesh(dae_ctx* ctx, int n_vert, const double* X, int n_tet, const int* tets,
                         const double* vmass, dae_material material, double E, double nu,
                         dae_mesh** out) {
    if (!ctx || !out) return DAE_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_vert <= 0 || n_tet <= 0 || !X || !tets || !vmass)
        return fail(ctx, DAE_ERR_INVALID_ARG, "empty mesh or missing arrays");
    if (!(nu > -1.0 && nu < 0.5) || !(E > 0))
        return fail(ctx, DAE_ERR_INVALID_ARG, "material parameters out of range");
    if (material != DAE_STVK && material != DAE_NEOHOOKEAN)
        return fail(ctx, DAE_ERR_INVALID_ARG, "bad material");
    CU(ctx, cudaSetDevice(ctx->device));
    // bring host copies for the precomputation
    std::vector<double> hX(3 * (size_t)n_vert), hm(n_vert);
    std::vector<int> ht(4 * (size_t)n_tet);
    CU(ctx, cudaMemcpy(hX.data(), X, hX.size() * sizeof(double), cudaMemcpyDefault));
    CU(ctx, cudaMemcpy(ht.data(), tets, ht.size() * sizeof(int), cudaMemcpyDefault));
    CU(ctx, cudaMemcpy(hm.data(), vmass, hm.size() * sizeof(double), cudaMemcpyDefault));
    std::vector<float> Bm(9 * (size_t)n_tet), vol(n_tet), mdof(3 * (size_t)n_vert);
    for (int e = 0; e < n_tet; ++e) {
        int v[4];
        for (int a = 0; a < 4; ++a) {
            v[a] = ht[4 * (size_t)e + a];
            if (v[a] < 0 || v[a] >= n_vert)
                return fail(ctx, DAE_ERR_INVALID_ARG, "tet %d vertex index %d out of range", e, v[a]);
        }
        double Dm[9];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) Dm[d * 3 + c] = hX[3 * v[c + 1] + d] - hX[3 * v[0] + d];
        double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                     Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
        if (!(std::fabs(det) > 0))
            return fail(ctx, DAE_ERR_INVALID_ARG, "tet %d is degenerate at rest", e);
        double inv[9];
        inv[0] = (Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det;
        inv[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
        inv[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
        inv[3] = (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det;
        inv[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
        inv[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
        inv[6] = (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det;
        inv[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
        inv[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
        for (int i = 0; i < 9; ++i) Bm[9 * (size_t)e + i] = (float)inv[i];
        vol[e] = (float)(std::fabs(det) / 6.0);
    }
    for (int v = 0; v < n_vert; ++v)
        for (int d = 0; d < 3; ++d) mdof[3 * (size_t)v + d] = (float)hm[v];
    dae_mesh* m = new dae_mesh();
    m->ctx = ctx;
    m->id = g_mesh_ids.fetch_add(1);
    m->n_vert = n_vert;
    m->n_tet = n_tet;
    m->material = material;
    m->mu = E / (2.0 * (1.0 + nu));
    m->lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    dae_status st = DAE_OK;
    if (!st) st = dmalloc(ctx, &m->X, hX.size());
    if (!st) st = dmalloc(ctx, &m->tets, ht.size());
    if (!st) st = dmalloc(ctx, &m->Bm, Bm.size());
    if (!st) st = dmalloc(ctx, &m->vol, vol.size());
    if (!st) st = dmalloc(ctx, &m->mdof, mdof.size());
    if (st) { dae_free_mesh(m); return st; }
    cudaMemcpy(m->X, hX.data(), hX.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(m->tets, ht.data(), ht.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(m->Bm, Bm.data(), Bm.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(m->vol, vol.data(), vol.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaError_t e = cudaMemcpy(m->mdof, mdof.data(), mdof.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { dae_free_mesh(m); return fail(ctx, DAE_ERR_CUDA, "mesh upload failed"); }
    *out = m;
    return DAE_OK;
}

dae_status dae_free_mesh(dae_mesh* m) {
    if (!m) return DAE_ERR_INVALID_ARG;
    cudaSetDevice(m->ctx->device);
    cudaStreamSynchronize(m->ctx->stream);
    dfree(m->X); dfree(m->tets); dfree(m->Bm); dfree(m->vol); dfree(m->mdof);
    delete m;
    return DAE_OK;
}

dae_status dae_decoder_set_cs_mode(dae_decoder* d, int exact) {
    if (!d) return DAE_ERR_INVALID_ARG;
    if (exact && (d->prec != DAE_FP32 || d->r > kMaxRExact || d->np > 0))
        return fail(d->ctx, DAE_ERR_UNSUPPORTED,
                    "the exact multicomplex activation runs in the FP32 form, r <= %d, no linear basis",
                    kMaxRExact);
    d->cs_exact = exact ? 1 : 0;
    return DAE_OK;
}

dae_status dae_eval_derivs(dae_ctx* ctx, const dae_decoder* dec_c, const double* q,
                           const double* qbar, const double* qbar_dot, double dt, float* u,
                           float* J, float* Hqq, float* dJ, float* Hw, float* Sdd) {
    TRY(check_common(ctx, dec_c, nullptr));
    dae_decoder* d = const_cast<dae_decoder*>(dec_c);
    if (!q || !qbar || !qbar_dot) return fail(ctx, DAE_ERR_INVALID_ARG, "q, qbar, qbar_dot required");
    if (!(dt > 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "dt must be > 0");
    const int r = d->r;
    const size_t N = d->N;
    Stage st(ctx);
    st.need(q, r * 8); st.need(u, N * 4); st.need(J, N * r * 4); st.need(Hqq, N * 4);
    st.need(dJ, N * r * 4); st.need(Hw, N * r * 4); st.need(Sdd, N * r * 4);
    TRY(st.reserve(st.plan));
    const double* dq;
    float *du, *dJo, *dHqq, *ddJ, *dHw, *dSdd;
    TRY(st.in(q, r, &dq));
    TRY(st.inout(u, N, &du, false));
    TRY(st.inout(J, N * r, &dJo, false));
    TRY(st.inout(Hqq, N, &dHqq, false));
    TRY(st.inout(dJ, N * r, &ddJ, false));
    TRY(st.inout(Hw, N * r, &dHw, false));
    TRY(st.inout(Sdd, N * r, &dSdd, false));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar, qbar, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar_dot, qbar_dot, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    const double h = std::ldexp(1.0, -20);
    Outs o;
    o.u = du; o.J = dJo; o.Hqq = dHqq; o.dJ = ddJ;
    const bool exact = d->cs_exact && d->prec == DAE_FP32;
    auto fwd = [&](int mode, const Outs& oo) {
        return exact ? enqueue_forward_exact(d, dq, dt, h, mode, oo)
                     : enqueue_forward(d, nullptr, dq, dt, h, mode, oo);
    };
    if (du || dJo || dHqq || ddJ) TRY(fwd(SEED_FULL, o));
    if (dHw) {
        Outs o2;
        o2.dJ = dHw;
        TRY(fwd(SEED_HW, o2));
    }
    if (dSdd) {
        Outs o3;
        o3.dJ = dSdd;
        TRY(fwd(SEED_SDD, o3));
    }
    TRY(st.finish());
    if (st.any_host) return check_device_status(ctx);
    return DAE_OK;
}

dae_status dae_assemble_reduced(dae_ctx* ctx, const dae_decoder* dec_c, const dae_mesh* m,
                                int n_cub, const int* cub_tets, const float* cub_w, const double* q,
                                const double* qbar, const double* qbar_dot, double dt,
                                const float* f_ext, double* phi, double* A, double* energy,
                                double* terms) {
    TRY(check_common(ctx, dec_c, m));
    if (!m) return fail(ctx, DAE_ERR_INVALID_ARG, "mesh required");
    dae_decoder* d = const_cast<dae_decoder*>(dec_c);
    if (!q || !qbar || !qbar_dot) return fail(ctx, DAE_ERR_INVALID_ARG, "q, qbar, qbar_dot required");
    if (!(dt > 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "dt must be > 0");
    TRY(validate_cub(ctx, m, n_cub, cub_tets, cub_w, d));
    const int r = d->np + d->r;   // system size
    Stage st(ctx);
    st.need(q, r * 8);
    TRY(st.reserve(st.plan));
    const double* dq;
    TRY(st.in(q, r, &dq));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar, qbar, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar_dot, qbar_dot, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    const int* dct = nullptr;
    const float* dcw = nullptr;
    TRY(stage_cubature(d, st, n_cub, cub_tets, cub_w, n_cub, &dct, &dcw));
    const float* dfe = nullptr;
    TRY(stage_fext(d, f_ext, &dfe));
    if (use_gram(d)) {
        TRY(ensure_gram(d, m));
        TRY(prepare_pext(d, dfe));
        TRY(prepare_gram_out(d, m, n_cub));
    }
    if (d->np > 0 && !gram_out(d, m))
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the linear subspace needs the Gram form (2K <= N)");
    EvalParams P;
    P.dt = dt; P.h = std::ldexp(1.0, -20); P.cub_tets = dct; P.cub_w = dcw; P.n_cub = n_cub;
    P.w_stride = 0; P.f_ext = dfe; P.control = 0; P.opts = nullptr; P.wnet = cub_w ? 0 : 1;
    TRY(enqueue_eval(d, m, nullptr, dq, P));
    const double* red = d->ws.red;
    const size_t rr = (size_t)r * r;
    if (phi) CU(ctx, cudaMemcpyAsync(phi, red, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    if (A) CU(ctx, cudaMemcpyAsync(A, red + r, rr * sizeof(double), cudaMemcpyDefault, ctx->stream));
    if (energy) CU(ctx, cudaMemcpyAsync(energy, red + r + rr, sizeof(double), cudaMemcpyDefault, ctx->stream));
    if (terms) CU(ctx, cudaMemcpyAsync(terms, red + r + rr + 1, (4 * rr + r) * sizeof(double),
                                       cudaMemcpyDefault, ctx->stream));
    bool host_out = (phi && !on_device(phi)) || (A && !on_device(A)) ||
                    (energy && !on_device(energy)) || (terms && !on_device(terms));
    TRY(st.finish());
    if (host_out || st.any_host) return check_device_status(ctx);
    return DAE_OK;
}

dae_status dae_newton_step(dae_ctx* ctx, const dae_decoder* dec_c, const dae_mesh* m, int n_cub,
                           const int* cub_tets, const float* cub_w, double* q, const double* qbar,
                           const double* qbar_dot, double dt, const float* f_ext,
                           const dae_newton_opts* opts_in, dae_newton_report* rep) {
    TRY(check_common(ctx, dec_c, m));
    if (!m) return fail(ctx, DAE_ERR_INVALID_ARG, "mesh required");
    dae_decoder* d = const_cast<dae_decoder*>(dec_c);
    if (!q || !qbar || !qbar_dot) return fail(ctx, DAE_ERR_INVALID_ARG, "q, qbar, qbar_dot required");
    if (!(dt > 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "dt must be > 0");
    TRY(validate_cub(ctx, m, n_cub, cub_tets, cub_w, d));
    dae_newton_opts opts;
    fill_opts(opts_in, &opts);
    if (opts.max_iter < 0 || opts.max_evals < 1 || opts.max_evals > 1000)
        return fail(ctx, DAE_ERR_INVALID_ARG, "bad Newton options");
    const int r = d->np + d->r;   // system size
    Stage st(ctx);
    st.need(q, r * 8);
    TRY(st.reserve(st.plan));
    double* dq;
    TRY(st.inout(q, r, &dq, true));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar, qbar, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CU(ctx, cudaMemcpyAsync(d->ws.qbar_dot, qbar_dot, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    const int* dct = nullptr;
    const float* dcw = nullptr;
    TRY(stage_cubature(d, st, n_cub, cub_tets, cub_w, n_cub, &dct, &dcw));
    const float* dfe = nullptr;
    TRY(stage_fext(d, f_ext, &dfe));
    if (use_gram(d)) {
        TRY(ensure_gram(d, m));
        TRY(prepare_pext(d, dfe));
        TRY(prepare_gram_out(d, m, n_cub));
    }
    if (d->np > 0 && !gram_out(d, m))
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the linear subspace needs the Gram form (2K <= N)");
    EvalParams P;
    P.dt = dt; P.h = opts.h_cs; P.cub_tets = dct; P.cub_w = dcw; P.n_cub = n_cub;
    P.w_stride = cub_w ? n_cub : 0; P.f_ext = dfe; P.control = 1; P.opts = &opts;
    P.wnet = cub_w ? 0 : 1;
    TRY(run_frames(d, m, P, 1, 1, 0, dq));
    CU(ctx, cudaMemcpyAsync(dq, d->ws.qout, r * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->last_ns = d->ws.hist;
    TRY(st.finish());
    if (rep) return dae_last_report(ctx, rep);
    return DAE_OK;
}

// Ties of a coupled step as given through the C ABI.
struct TieSpec {
    int n_pairs; const int* pairs; int n_anch; const int* anch; double kc;
};

// The grouped Newton step of n_sys systems: independent (spec == nullptr, per-system
// reports in reps) or coupled by ties (one global report in grep).
static dae_status grouped_step(dae_ctx* ctx, int n_sys, const dae_system* sys, double dt,
                               const dae_newton_opts* opts_in, dae_newton_report* reps,
                               const TieSpec* spec, dae_newton_report* grep) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    if (n_sys < 0 || (n_sys > 0 && !sys)) return fail(ctx, DAE_ERR_INVALID_ARG, "bad system list");
    if (n_sys == 0) return DAE_OK;
    if (!(dt > 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "dt must be > 0");
    dae_newton_opts opts;
    fill_opts(opts_in, &opts);
    if (opts.max_iter < 0 || opts.max_evals < 1 || opts.max_evals > 1000)
        return fail(ctx, DAE_ERR_INVALID_ARG, "bad Newton options");
    std::vector<dae_decoder*> ds(n_sys);
    std::vector<const dae_mesh*> ms(n_sys);
    std::vector<int> ncub(n_sys), hasf(n_sys), pred(n_sys);
    std::vector<const dae_decoder*> seen;
    for (int i = 0; i < n_sys; ++i) {
        const dae_system& y = sys[i];
        TRY(check_common(ctx, y.dec, y.mesh));
        if (!y.mesh) return fail(ctx, DAE_ERR_INVALID_ARG, "system %d: mesh required", i);
        if (!y.q || !y.qbar || !y.qbar_dot)
            return fail(ctx, DAE_ERR_INVALID_ARG, "system %d: q, qbar, qbar_dot required", i);
        TRY(validate_cub(ctx, y.mesh, y.n_cub, y.cub_tets, y.cub_w, y.dec));
        dae_decoder* d = const_cast<dae_decoder*>(y.dec);
        if (d->prec == DAE_FP32 || !d->ws.chain_ok || !d->layers[0].tmR_ok)
            return fail(ctx, DAE_ERR_UNSUPPORTED, "system %d: the grouped step needs a tensor-core precision", i);
        if (d->prec != sys[0].dec->prec)
            return fail(ctx, DAE_ERR_INVALID_ARG, "system %d: all decoders must share one precision", i);
        if (d->L < 2) return fail(ctx, DAE_ERR_UNSUPPORTED, "system %d: a decoder needs a hidden layer", i);
        ds[i] = d;
        ms[i] = y.mesh;
        ncub[i] = y.n_cub;
        hasf[i] = y.f_ext ? 1 : 0;
        pred[i] = (!y.cub_w && y.n_cub > 0) ? 1 : 0;
        seen.push_back(y.dec);
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return fail(ctx, DAE_ERR_INVALID_ARG, "a decoder appears in two systems (its workspace is per decoder)");
    std::unique_ptr<Coupling> topo;
    if (spec) {
        std::vector<int> rr(n_sys), nv(n_sys);
        for (int i = 0; i < n_sys; ++i) {
            if (ds[i]->np > 0) return fail(ctx, DAE_ERR_UNSUPPORTED, "system %d: a linear subspace in a coupled step", i);
            rr[i] = ds[i]->r;
            nv[i] = ms[i]->n_vert;
        }
        topo.reset(new Coupling());
        TRY(build_topology(ctx, *topo, rr, nv, spec->n_pairs, spec->pairs, spec->n_anch, spec->anch));
        topo->kc = spec->kc;
    }
    // per-system set-up that is cached across calls
    for (int i = 0; i < n_sys; ++i) {
        // (coupled: room for the tie forces after the cubature pairs of W_L^T a)
        TRY(ensure_cubature(ds[i], ncub[i] + (topo ? topo->ntv_dom[i] : 0), ncub[i]));
        Workspace& wi = ds[i]->ws;
        if (pred[i] && wi.wn_cap < ncub[i]) {
            dfree(wi.wn_w);
            TRY(dmalloc(ctx, &wi.wn_w, (size_t)ncub[i]));
            wi.wn_cap = ncub[i];
        }
        if (use_gram(ds[i])) {
            TRY(ensure_gram(ds[i], ms[i]));
            TRY(ensure_gs(ds[i], ms[i], ncub[i]));
        }
        if (ds[i]->np > 0 && !gram_out(ds[i], ms[i]))
            return fail(ctx, DAE_ERR_UNSUPPORTED, "system %d: the linear subspace needs the Gram form", i);
    }
    void*& slot = spec ? ctx->batch_coupled : ctx->batch;
    BatchPlan* b = (BatchPlan*)slot;
    if (!b) {
        b = new BatchPlan();
        slot = b;
        CU(ctx, cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming));
    }
    for (int i = 0; i < n_sys; ++i)
        if (hasf[i] && use_gram(ds[i])) TRY(ensure_pext_bufs(ds[i]));
    std::vector<BatchKey> key(n_sys);
    for (int i = 0; i < n_sys; ++i) {
        const Workspace& w = ds[i]->ws;
        key[i] = BatchKey{ds[i]->id, ms[i]->id, w.cub_tets, w.cub_w, w.fe_w, w.G, w.pext,
                          gram_out(ds[i], ms[i]) ? (w.Gs32 ? (const void*)w.Gs32 : (const void*)w.Gsh) : nullptr,
                          pred[i] ? (const void*)w.wn_w : nullptr, ncub[i], hasf[i]};
    }
    bool same = b->gexec && b->n == n_sys && b->dt == dt && b->prec == (int)ds[0]->prec &&
                memcmp(&b->opts, &opts, sizeof opts) == 0 &&
                memcmp(b->key.data(), key.data(), n_sys * sizeof(BatchKey)) == 0;
    if (spec)
        same = same && b->cpl && b->cpl->kc == topo->kc && b->cpl->pairs == topo->pairs &&
               b->cpl->anchors == topo->anchors;
    if (!same) {
        if (spec) {
            delete b->cpl;
            b->cpl = topo.release();
        }
        TRY(build_batch(ctx, b, ds, ms, ncub, hasf, pred, dt, opts));
        b->key = key;
        b->n = n_sys;
        b->dt = dt;
        b->prec = (int)ds[0]->prec;
        b->opts = opts;
    }
    if (b->epoch != ctx->timeout_epoch) {
        CU(ctx, cudaMemsetAsync(b->gb, 0, sizeof(GridBar), ctx->stream));
        b->epoch = ctx->timeout_epoch;
    }
    // inputs into the systems' workspaces and the results out: host arrays through one
    // pinned buffer and one upload (with the copy lists), then one grouped device copy
    // each way
    struct HostIn { const void* src; size_t n; void* dst; };
    std::vector<CopyDesc> cin, cout;
    std::vector<HostIn> hin;
    size_t hbytes = 0;
    auto add = [&](const void* src, void* dst, size_t nb) {
        if (!src || nb == 0) return;
        if (on_device(src)) {
            cin.push_back(CopyDesc{src, dst, (unsigned long long)nb});
        } else {
            hin.push_back(HostIn{src, nb, dst});
            hbytes += round_up(nb, 16);
        }
    };
    std::vector<int> host_q;
    for (int i = 0; i < n_sys; ++i) {
        const dae_system& y = sys[i];
        Workspace& w = ds[i]->ws;
        const int r = ds[i]->np + ds[i]->r;   // system size
        add(y.q, b->q0 + (size_t)i * kMaxR, r * sizeof(double));
        add(y.qbar, w.qbar, r * sizeof(double));
        add(y.qbar_dot, w.qbar_dot, r * sizeof(double));
        add(y.cub_tets, w.cub_tets, (size_t)ncub[i] * sizeof(int));
        add(y.cub_w, w.cub_w, (size_t)ncub[i] * sizeof(float));
        add(y.f_ext, w.f_ext, (size_t)ds[i]->N * sizeof(float));
        if (on_device(y.q))
            cout.push_back(CopyDesc{b->qout + (size_t)i * kMaxR, y.q, (unsigned long long)(r * sizeof(double))});
        else
            host_q.push_back(i);
        if (reps) cout.push_back(CopyDesc{w.ns, b->ns_out + i, (unsigned long long)sizeof(NewtonState)});
    }
    const size_t n_in = hin.size() + cin.size();
    const size_t o_cin = hbytes, o_cout = round_up(o_cin + n_in * sizeof(CopyDesc), 16);
    const size_t total = o_cout + cout.size() * sizeof(CopyDesc);
    Stage stg(ctx);
    TRY(stg.reserve(total));
    CU(ctx, cudaEventSynchronize(b->staged));   // the previous call's upload has completed
    TRY(ensure_pinned(ctx, total));
    char* P = (char*)ctx->pinned;
    char* D = (char*)ctx->dstage;
    size_t o = 0;
    for (const HostIn& h : hin) {
        memcpy(P + o, h.src, h.n);
        cin.push_back(CopyDesc{D + o, h.dst, (unsigned long long)h.n});
        o += round_up(h.n, 16);
    }
    memcpy(P + o_cin, cin.data(), cin.size() * sizeof(CopyDesc));
    memcpy(P + o_cout, cout.data(), cout.size() * sizeof(CopyDesc));
    CU(ctx, cudaMemcpyAsync(D, P, total, cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaEventRecord(b->staged, ctx->stream));
    ctx->launches += 2;
    launch_copy_batch(ctx->stream, (const CopyDesc*)(D + o_cin), (int)cin.size());
    if (b->max_gather > 0) {
        // the stacked Gram operands' cubature rows from the staged tets
        GatherArgs gmax;
        memset(&gmax, 0, sizeof gmax);
        gmax.n_rows = b->max_gather;
        ctx->launches += 1;
        launch_gather_cub_rows(ctx->stream, b->gather, gmax, n_sys);
    }
    for (int i = 0; i < n_sys; ++i)
        if (hasf[i] && use_gram(ds[i])) TRY(prepare_pext(ds[i], ds[i]->ws.f_ext));
    if (ctx->prof_on) {
        // explicit launches (timed phases): the host reads the any-running flag after
        // every evaluation
        ctx->launches += b->cpl ? 3 : 2;
        launch_frame_begin_batched(ctx->stream, b->frame, n_sys, 0, 0);
        if (b->cpl) launch_coupled_begin(ctx->stream, b->cpl->args);
        for (int e = 0; e < opts.max_evals; ++e) {
            TRY(enqueue_batch_eval(ctx, b, ds[0]->prec, 0, b->flag));
            int run = 0;
            CU(ctx, cudaMemcpyAsync(&run, b->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CU(ctx, cudaStreamSynchronize(ctx->stream));
            if (!run) break;
        }
        launch_frame_end_batched(ctx->stream, b->frame, n_sys);
    } else {
        CU(ctx, cudaGraphLaunch(b->gexec, ctx->stream));
    }
    launch_copy_batch(ctx->stream, (const CopyDesc*)(D + o_cout), (int)cout.size());
    ctx->last_ns = ds[n_sys - 1]->ws.ns;
    std::vector<NewtonState> hs;
    if (!host_q.empty() || reps) {
        std::vector<double> qh;
        if (!host_q.empty()) {
            qh.resize((size_t)n_sys * kMaxR);
            CU(ctx, cudaMemcpyAsync(qh.data(), b->qout, qh.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (reps) {
            hs.resize(n_sys);
            CU(ctx, cudaMemcpyAsync(hs.data(), b->ns_out, n_sys * sizeof(NewtonState), cudaMemcpyDeviceToHost, ctx->stream));
        }
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        for (int i : host_q)
            memcpy(sys[i].q, qh.data() + (size_t)i * kMaxR, (ds[i]->np + ds[i]->r) * sizeof(double));
    }
    CU(ctx, cudaGetLastError());
    if (reps) {
        TRY(check_device_status(ctx));
        int worst = -1;
        for (int i = 0; i < n_sys; ++i) {
            to_report(hs[i], &reps[i]);
            if (hs[i].status && worst < 0) worst = i;
        }
        if (worst >= 0)
            return fail(ctx, (dae_status)hs[worst].status, "system %d failed: %s", worst,
                        dae_status_string((dae_status)hs[worst].status));
    }
    if (grep) {
        CoupledState cs;
        CU(ctx, cudaMemcpyAsync(&cs, b->cpl->cs, sizeof cs, cudaMemcpyDeviceToHost, ctx->stream));
        TRY(check_device_status(ctx));
        grep->iters = cs.iters;
        grep->evals = cs.evals;
        grep->converged = cs.converged;
        grep->status = cs.status;
        grep->phi_norm0 = cs.phi_norm0;
        grep->phi_norm = std::sqrt(cs.merit_acc);
        grep->energy = cs.energy;
        grep->alpha = cs.alpha;
        grep->full_evals = cs.nfull;
        if (cs.status) return fail(ctx, (dae_status)cs.status, "coupled step failed: %s",
                                   dae_status_string((dae_status)cs.status));
    }
    return DAE_OK;
}

dae_status dae_newton_step_batched(dae_ctx* ctx, int n_sys, const dae_system* sys, double dt,
                                   const dae_newton_opts* opts, dae_newton_report* reps) {
    return grouped_step(ctx, n_sys, sys, dt, opts, reps, nullptr, nullptr);
}

dae_status dae_newton_step_coupled(dae_ctx* ctx, int n_sys, const dae_system* sys, int n_pairs,
                                   const int* pairs, int n_anchors, const int* anchors, double k_c,
                                   double dt, const dae_newton_opts* opts, dae_newton_report* rep) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    if (n_pairs < 0 || n_anchors < 0 || (n_pairs > 0 && !pairs) || (n_anchors > 0 && !anchors))
        return fail(ctx, DAE_ERR_INVALID_ARG, "tie pairs / anchors missing");
    if ((n_pairs > 0 && on_device(pairs)) || (n_anchors > 0 && on_device(anchors)))
        return fail(ctx, DAE_ERR_INVALID_ARG, "tie pairs and anchors must be host arrays");
    if (!(k_c >= 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "k_c must be >= 0");
    if (n_sys < 1) return fail(ctx, DAE_ERR_INVALID_ARG, "no systems");
    const TieSpec spec{n_pairs, pairs, n_anchors, anchors, k_c};
    dae_newton_report tmp;
    return grouped_step(ctx, n_sys, sys, dt, opts, nullptr, &spec, rep ? rep : &tmp);
}

dae_status dae_last_report(dae_ctx* ctx, dae_newton_report* rep) {
    if (!ctx || !rep) return DAE_ERR_INVALID_ARG;
    if (!ctx->last_ns) return fail(ctx, DAE_ERR_INVALID_ARG, "no Newton step has run");
    NewtonState s;
    CU(ctx, cudaMemcpyAsync(&s, ctx->last_ns, sizeof s, cudaMemcpyDeviceToHost, ctx->stream));
    TRY(check_device_status(ctx));
    to_report(s, rep);
    if (s.status != 0) return fail(ctx, (dae_status)s.status, "Newton frame failed: %s", dae_status_string((dae_status)s.status));
    return DAE_OK;
}

dae_status dae_rollout(dae_ctx* ctx, const dae_decoder* dec_c, const dae_mesh* m, int n_cub,
                       const int* cub_tets, const float* cub_w, int n_frames, double* q,
                       double* qdot, double dt, const float* f_ext, const dae_newton_opts* opts_in,
                       double* q_traj, dae_newton_report* reports) {
    TRY(check_common(ctx, dec_c, m));
    if (!m) return fail(ctx, DAE_ERR_INVALID_ARG, "mesh required");
    dae_decoder* d = const_cast<dae_decoder*>(dec_c);
    if (!q || !qdot || n_frames < 0) return fail(ctx, DAE_ERR_INVALID_ARG, "q, qdot required, n_frames >= 0");
    if (!(dt > 0)) return fail(ctx, DAE_ERR_INVALID_ARG, "dt must be > 0");
    TRY(validate_cub(ctx, m, n_cub, cub_tets, cub_w, d));
    dae_newton_opts opts;
    fill_opts(opts_in, &opts);
    const int r = d->np + d->r;   // system size
    Stage st(ctx);
    Workspace& w = d->ws;
    TRY(ensure_frames(d, n_frames));
    // the state straight into the frame state and back (host or device memory alike)
    CU(ctx, cudaMemcpyAsync(w.qbar, q, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CU(ctx, cudaMemcpyAsync(w.qbar_dot, qdot, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    const int* dct = nullptr;
    const float* dcw = nullptr;
    TRY(stage_cubature(d, st, n_cub, cub_tets, cub_w, n_cub * n_frames, &dct, &dcw));
    const float* dfe = nullptr;
    TRY(stage_fext(d, f_ext, &dfe));
    if (use_gram(d)) {
        TRY(ensure_gram(d, m));
        TRY(prepare_pext(d, dfe));
        TRY(prepare_gram_out(d, m, n_cub));
    }
    if (d->np > 0 && !gram_out(d, m))
        return fail(ctx, DAE_ERR_UNSUPPORTED, "the linear subspace needs the Gram form (2K <= N)");
    EvalParams P;
    P.dt = dt; P.h = opts.h_cs; P.cub_tets = dct; P.cub_w = dcw; P.n_cub = n_cub;
    P.w_stride = cub_w ? n_cub : 0; P.f_ext = dfe; P.control = 1; P.opts = &opts;
    P.wnet = cub_w ? 0 : 1;
    if (n_frames > 0) TRY(run_frames(d, m, P, n_frames, 0, 1, nullptr));
    CU(ctx, cudaGetLastError());
    CU(ctx, cudaMemcpyAsync(q, w.qbar, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CU(ctx, cudaMemcpyAsync(qdot, w.qbar_dot, r * sizeof(double), cudaMemcpyDefault, ctx->stream));
    if (q_traj && n_frames > 0)
        CU(ctx, cudaMemcpyAsync(q_traj, w.traj, (size_t)n_frames * r * sizeof(double),
                                cudaMemcpyDefault, ctx->stream));
    ctx->last_ns = n_frames > 0 ? w.hist + (n_frames - 1) : nullptr;
    if (!(reports && n_frames > 0)) {
        // host outputs are complete when the call returns (device ones stay asynchronous)
        if (!on_device(q) || !on_device(qdot) || (q_traj && !on_device(q_traj)))
            CU(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (reports && n_frames > 0) {
        std::vector<NewtonState> hs(n_frames);
        CU(ctx, cudaMemcpyAsync(hs.data(), w.hist, n_frames * sizeof(NewtonState),
                                cudaMemcpyDeviceToHost, ctx->stream));
        TRY(check_device_status(ctx));   // one wait for every copy above
        int worst = 0;
        for (int f = 0; f < n_frames; ++f) {
            to_report(hs[f], &reports[f]);
            if (hs[f].status && !worst) worst = hs[f].status;
        }
        if (worst) return fail(ctx, (dae_status)worst, "a rollout frame failed: %s", dae_status_string((dae_status)worst));
    }
    return DAE_OK;
}

dae_status dae_profile_enable(dae_ctx* ctx, unsigned mask) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    ctx->prof_on = mask;
    return DAE_OK;
}

dae_status dae_profile_read(dae_ctx* ctx, double* ms, long long* count) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    CU(ctx, cudaSetDevice(ctx->device));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<double> acc(DAE_N_PHASES, 0.0);
    std::vector<long long> cnt(DAE_N_PHASES, 0);
    for (auto& rec : ctx->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, rec.a, rec.b) == cudaSuccess) {
            acc[rec.phase] += t;
            cnt[rec.phase] += 1;
        }
        ctx->ev_pool.push_back(rec.a);
        ctx->ev_pool.push_back(rec.b);
    }
    cudaGetLastError();
    ctx->recs.clear();
    for (int i = 0; i < DAE_N_PHASES; ++i) {
        if (ms) ms[i] = acc[i];
        if (count) count[i] = cnt[i];
    }
    return DAE_OK;
}

dae_status dae_selftest_bounded_waits(dae_ctx* ctx) {
    if (!ctx) return DAE_ERR_INVALID_ARG;
    CU(ctx, cudaSetDevice(ctx->device));
    GridBar* gb = nullptr;
    int* out = nullptr;
    const int nb = 2;
    TRY(dmalloc(ctx, &gb, 1));
    TRY(dmalloc(ctx, &out, nb));
    ctx->launches += 1;
    if (run_wait_selftest(ctx->stream, gb, out, nb)) {
        dfree(gb); dfree(out);
        return fail(ctx, DAE_ERR_CUDA, "self-test launch failed");
    }
    int h[nb] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(gb); dfree(out);
    if (e != cudaSuccess) return fail(ctx, DAE_ERR_CUDA, "self-test: %s", cudaGetErrorString(e));
    for (int i = 0; i < nb; ++i)
        if (h[i] != 1) return fail(ctx, DAE_ERR_TIMEOUT, "a bounded wait did not give up as expected");
    return DAE_OK;
}

long long dae_launch_count(const dae_ctx* ctx) {
    if (!ctx) return -1;
    unsigned long long k = 0;
    cudaSetDevice(ctx->device);
    if (cudaMemcpyAsync(&k, ctx->d_kcount, sizeof k, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return ctx->launches + (long long)k;
}

}  // extern "C"
