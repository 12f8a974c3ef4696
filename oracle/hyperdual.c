/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library: it evaluates the
 * plain definitions with exact forward-mode hyper-dual numbers (three nilpotent
 * units e1, e2, e3 with e_k^2 = 0), not with complex steps.
 *
 * A hyper-dual number holds 8 components indexed by the subset of units it
 * multiplies: [0]=1 [1]=e1 [2]=e2 [3]=e1e2 [4]=e3 [5]=e1e3 [6]=e2e3 [7]=e1e2e3.
 * For f(x0 + e1 s1 + e2 s2 + e3 s3) the components are the derivatives of f in
 * the seeded directions: [1] = Df[s1], [3] = D2f[s1,s2], [7] = D3f[s1,s2,s3].
 * This is what the paper's multicomplex perturbations approximate (Sec. 4.1,
 * Eqs. 13-17): the i-unit components of a multicomplex step divided by h^k
 * equal these components up to O(h^2).
 *
 * Contents
 *   orc_act_jet       -- hidden activation applied to one jet (tanh, sin, linear;
 *                        sin is the paper's choice, Sec. 3.5)
 *   orc_decoder_jets  -- u = D(q) of the fully connected decoder (Sec. 3.5,
 *                        Fig. 3) with its seeded derivatives, for a batch of seed
 *                        triples (OpenMP over the batch)
 *   orc_tet_fk        -- StVK / Neo-Hookean tet energy, force (gradient) and
 *                        12x12 stiffness (Hessian) by hyper-dual differentiation
 *                        of V_e * Psi(F) (Sec. 5: f_int at cubature elements)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double c[8]; } hd;

static hd hd_const(double v) { hd r; memset(&r, 0, sizeof r); r.c[0] = v; return r; }

static hd hd_add(hd x, hd y) { hd r; for (int m = 0; m < 8; ++m) r.c[m] = x.c[m] + y.c[m]; return r; }
static hd hd_sub(hd x, hd y) { hd r; for (int m = 0; m < 8; ++m) r.c[m] = x.c[m] - y.c[m]; return r; }
static hd hd_scale(hd x, double s) { hd r; for (int m = 0; m < 8; ++m) r.c[m] = x.c[m] * s; return r; }

/* Product: component m collects x[s] * y[m \ s] over all subsets s of m
 * (units are nilpotent, so overlapping subsets vanish). */
static hd hd_mul(hd x, hd y) {
    hd r;
    for (int m = 0; m < 8; ++m) {
        double acc = 0.0;
        for (int s = 0; s < 8; ++s)
            if ((s & m) == s) acc += x.c[s] * y.c[m ^ s];
        r.c[m] = acc;
    }
    return r;
}

/* f(x0 + d) = f(x0) + f'(x0) d + f''(x0) d^2/2 + f'''(x0) d^3/6 (d nilpotent of
 * order 3, so the Taylor series terminates exactly). */
static hd hd_apply(hd x, double f0, double f1, double f2, double f3) {
    hd d = x; d.c[0] = 0.0;
    hd d2 = hd_mul(d, d), d3 = hd_mul(d2, d);
    hd r = hd_const(f0);
    r = hd_add(r, hd_scale(d, f1));
    r = hd_add(r, hd_scale(d2, f2 / 2.0));
    r = hd_add(r, hd_scale(d3, f3 / 6.0));
    return r;
}

enum { ORC_TANH = 0, ORC_SIN = 1, ORC_LINEAR = 2 };

static hd hd_act(int act, hd x) {
    double a = x.c[0];
    if (act == ORC_TANH) {
        double t = tanh(a), t1 = 1.0 - t * t;
        return hd_apply(x, t, t1, -2.0 * t * t1, -2.0 * t1 * (1.0 - 3.0 * t * t));
    } else if (act == ORC_SIN) {
        double s = sin(a), c = cos(a);
        return hd_apply(x, s, c, -s, -c);
    }
    return x;
}

static hd hd_log(hd x) {
    double a = x.c[0];
    return hd_apply(x, log(a), 1.0 / a, -1.0 / (a * a), 2.0 / (a * a * a));
}

/* Hidden activation on one jet (8 components in, 8 out). */
void orc_act_jet(int act, const double* in, double* out) {
    hd x; memcpy(x.c, in, sizeof x.c);
    hd y = hd_act(act, x);
    memcpy(out, y.c, sizeof y.c);
}

/*
 * Decoder jets.  Layers l = 0..n_run-1 compute z = W_l a + b_l with W_l
 * row-major (widths[l+1] x widths[l]); every layer but the last one of the
 * whole decoder (index n_layers-1) applies the hidden activation.  The input is
 * the jet q + e1 s1 + e2 s2 + e3 s3.
 *
 * n_seed jobs are evaluated; job k reads seeds s1,s2,s3 at offset k*r (a NULL
 * seed array means zero).  If n_run == n_layers the outputs are the decoder
 * rows listed in rows[0..n_rows) (rows == NULL: all rows, n_rows ignored);
 * otherwise the outputs are all widths[n_run] activations after layer n_run.
 * out is (n_seed, n_out_rows, 8).  Returns 0, or -1 on bad arguments.
 */
int orc_decoder_jets(int n_layers, const int* widths, const float* const* W,
                     const float* const* b, int act, int n_run,
                     const double* q, int n_seed, const double* s1, const double* s2,
                     const double* s3, int n_rows, const int* rows, double* out) {
    if (n_layers < 1 || n_run < 1 || n_run > n_layers || n_seed < 0) return -1;
    const int r = widths[0];
    int wmax = 0;
    for (int l = 0; l <= n_layers; ++l) if (widths[l] > wmax) wmax = widths[l];
    const int last = (n_run == n_layers);
    const int n_out = last ? (rows ? n_rows : widths[n_layers]) : widths[n_run];
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n_seed; ++k) {
        hd* a = (hd*)malloc(sizeof(hd) * (size_t)wmax);
        hd* z = (hd*)malloc(sizeof(hd) * (size_t)wmax);
        if (!a || !z) { free(a); free(z); fail = 1; continue; }
        for (int i = 0; i < r; ++i) {
            a[i] = hd_const(q[i]);
            a[i].c[1] = s1 ? s1[(size_t)k * r + i] : 0.0;
            a[i].c[2] = s2 ? s2[(size_t)k * r + i] : 0.0;
            a[i].c[4] = s3 ? s3[(size_t)k * r + i] : 0.0;
        }
        for (int l = 0; l < n_run; ++l) {
            const int n_in = widths[l], n_o = widths[l + 1];
            const int is_out_layer = (l == n_layers - 1);
            const int cnt = (is_out_layer && rows) ? n_rows : n_o;
            for (int ii = 0; ii < cnt; ++ii) {
                const int i = (is_out_layer && rows) ? rows[ii] : ii;
                const float* wr = W[l] + (size_t)i * n_in;
                hd acc = hd_const((double)b[l][i]);
                for (int j = 0; j < n_in; ++j) {
                    const double w = (double)wr[j];
                    for (int m = 0; m < 8; ++m) acc.c[m] += w * a[j].c[m];
                }
                z[ii] = is_out_layer ? acc : hd_act(act, acc);
            }
            hd* t = a; a = z; z = t;
        }
        double* o = out + (size_t)k * n_out * 8;
        for (int i = 0; i < n_out; ++i) memcpy(o + (size_t)i * 8, a[i].c, 8 * sizeof(double));
        free(a); free(z);
    }
    return fail ? -2 : 0;
}

/* ---------------------------------------------------------------- tet FEM -- */

/* Energy V_e * Psi(F) of one tet as a jet of its 12 nodal positions x (node-major
 * x0,y0,z0,x1,...).  Dm = [X1-X0, X2-X0, X3-X0], F = Ds Dm^{-1}, V_e = |det Dm|/6.
 *   StVK:         E = (F^T F - I)/2,  Psi = mu tr(E^2) + lam/2 (tr E)^2
 *   Neo-Hookean:  Psi = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2,  J = det F
 */
enum { ORC_STVK = 0, ORC_NEOHOOKEAN = 1 };

static int tet_energy(const double* X, const hd* x, int mat, double mu, double lam, hd* out) {
    double Dm[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) Dm[d][c] = X[3 * (c + 1) + d] - X[d];
    double det = Dm[0][0] * (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1])
               - Dm[0][1] * (Dm[1][0] * Dm[2][2] - Dm[1][2] * Dm[2][0])
               + Dm[0][2] * (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]);
    if (det == 0.0) return -1;
    double Bm[3][3];
    Bm[0][0] = (Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1]) / det;
    Bm[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
    Bm[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
    Bm[1][0] = (Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2]) / det;
    Bm[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
    Bm[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
    Bm[2][0] = (Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0]) / det;
    Bm[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
    Bm[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
    const double V = fabs(det) / 6.0;

    hd Ds[3][3], F[3][3];
    for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) Ds[d][c] = hd_sub(x[3 * (c + 1) + d], x[d]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            hd acc = hd_const(0.0);
            for (int k = 0; k < 3; ++k) acc = hd_add(acc, hd_scale(Ds[i][k], Bm[k][j]));
            F[i][j] = acc;
        }
    hd psi;
    if (mat == ORC_STVK) {
        hd E[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                hd acc = hd_const(0.0);
                for (int k = 0; k < 3; ++k) acc = hd_add(acc, hd_mul(F[k][i], F[k][j]));
                if (i == j) acc.c[0] -= 1.0;
                E[i][j] = hd_scale(acc, 0.5);
            }
        hd trE2 = hd_const(0.0), trE = hd_const(0.0);
        for (int i = 0; i < 3; ++i) {
            trE = hd_add(trE, E[i][i]);
            for (int j = 0; j < 3; ++j) trE2 = hd_add(trE2, hd_mul(E[i][j], E[j][i]));
        }
        psi = hd_add(hd_scale(trE2, mu), hd_scale(hd_mul(trE, trE), 0.5 * lam));
    } else {
        hd I1 = hd_const(0.0);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) I1 = hd_add(I1, hd_mul(F[i][j], F[i][j]));
        hd J = hd_sub(hd_add(hd_mul(F[0][0], hd_sub(hd_mul(F[1][1], F[2][2]), hd_mul(F[1][2], F[2][1]))),
                             hd_mul(F[0][2], hd_sub(hd_mul(F[1][0], F[2][1]), hd_mul(F[1][1], F[2][0])))),
                      hd_mul(F[0][1], hd_sub(hd_mul(F[1][0], F[2][2]), hd_mul(F[1][2], F[2][0]))));
        if (!(J.c[0] > 0.0)) return -7;
        hd lnJ = hd_log(J);
        I1.c[0] -= 3.0;
        psi = hd_add(hd_sub(hd_scale(I1, 0.5 * mu), hd_scale(lnJ, mu)),
                     hd_scale(hd_mul(lnJ, lnJ), 0.5 * lam));
    }
    *out = hd_scale(psi, V);
    return 0;
}

/*
 * One tet: X, x are the 12 rest / deformed nodal coordinates (node-major).
 * energy = V_e Psi, f[a] = d(V_e Psi)/dx_a, K[a*12+b] = d2(V_e Psi)/dx_a dx_b.
 * Returns 0, -1 for a degenerate rest tet, -7 for an inverted Neo-Hookean tet.
 */
int orc_tet_fk(const double* X, const double* x, int mat, double mu, double lam,
               double* energy, double* f, double* K) {
    hd xs[12], e;
    for (int a = 0; a < 12; ++a) xs[a] = hd_const(x[a]);
    int st = tet_energy(X, xs, mat, mu, lam, &e);
    if (st) return st;
    *energy = e.c[0];
    for (int a = 0; a < 12; ++a) {
        xs[a].c[1] = 1.0;
        if (f) {
            st = tet_energy(X, xs, mat, mu, lam, &e);
            if (st) return st;
            f[a] = e.c[1];
        }
        if (K) {
            for (int bb = a; bb < 12; ++bb) {
                xs[bb].c[2] = 1.0;
                st = tet_energy(X, xs, mat, mu, lam, &e);
                xs[bb].c[2] = 0.0;
                if (st) return st;
                K[a * 12 + bb] = e.c[3];
                K[bb * 12 + a] = e.c[3];
            }
        }
        xs[a].c[1] = 0.0;
    }
    return 0;
}

/* Batched over tets: X, x are (n, 12); energy (n), f (n, 12), K (n, 144);
 * status (n) receives each tet's return code. */
void orc_tets_fk(int n, const double* X, const double* x, int mat, double mu, double lam,
                 double* energy, double* f, double* K, int* status) {
#pragma omp parallel for schedule(static)
    for (int e = 0; e < n; ++e)
        status[e] = orc_tet_fk(X + 12 * (size_t)e, x + 12 * (size_t)e, mat, mu, lam,
                               energy + e, f ? f + 12 * (size_t)e : 0,
                               K ? K + 144 * (size_t)e : 0);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
