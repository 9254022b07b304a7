/*
 * FP64 CPU oracle for the FWIME operators -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Barnier et al., "Full waveform inversion by model
 * extension: practical applications", Theory section):
 *   f(m)          nonlinear forward (acoustic, isotropic, constant density, Eq. 1)
 *   B(m), B*(m)   non-extended Born and its adjoint (Eq. 8)
 *   B~(m), B~*    Born extended with horizontal subsurface offsets and its
 *                 adjoint, the extended imaging condition (Eq. 1, Eq. 2)
 *   T(m,p~), T*   data-space tomographic operator and adjoint (Eq. 9)
 *   grad, Phi     the FWIME objective at fixed p~ and its gradient
 *                 B* r + T* r with r = f + B~ p~ - d (Eq. 1, Eqs. 7-9), S = I.
 *
 * The paper defers every discretisation detail to a companion paper, so this
 * file implements one explicit discrete reading, used identically by the GPU
 * path (see the "Readings" list in the design notes):
 *   grid   physical nz x nx, sponge W points, plus a 4-point zero halo;
 *          padded NZ = nz + 2(W+4), NX = nx + 2(W+4); "active" points are
 *          4 <= IZ < NZ-4, 4 <= IX < NX-4, fields are 0 elsewhere.
 *   L      8th-order central Laplacian, coefficients -205/72, 8/5, -1/5,
 *          8/315, -1/560, applied at active points.
 *   sponge gamma = g1(kz) g1(kx), k = points outside the physical region,
 *          g1(k) = exp(-(0.3 k / W)^2)   (Cerjan-type taper, Marmousi2 section).
 *   step   q^{n+1} = gamma (2 q^n - gamma q^{n-1} + c (L q^n + s^n)),
 *          c = v^2 dt^2 (v edge-replicated into the padding), q^{-1}=q^0=0,
 *          n = 0..nt-2; point source s^n = w[n]/(dx dz); record d[n]=q^n(rec).
 *   D2t    D^n = (q^{n+1} - 2 q^n + q^{n-1})/dt^2, n = 0..nt-2.
 *   Born   secondary source b dv D2t q0, b = 2/v^3 (d c / d v = c b v).
 *   ext.   e^n(y) = sum_h W(y-h,h) D^n(y-2h), W = b p~, h along x, nh odd,
 *          terms whose points leave the active region dropped.
 *   fs     (fs = 1) the top physical row is a pressure-release surface: after every
 *          step q = 0 there and the 4 rows above hold the odd mirror -q of the 4
 *          rows below (the projection M); rows further up are inactive.
 *   lags   (lag > 0) e^n(x) = sum_i W(x,i) D^{n-2 s_i}(x), s_i = (i-hm) lag, D^m = 0
 *          outside 0 <= m <= nt-2: lag tau couples the source side at t - tau
 *          with the receiver side at t + tau.
 *   adj.   the literal transpose of each primitive, composed in reverse.
 * Everything is double precision, sequential loops, no reordering of sums
 * beyond the loop order written here (compile with -ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nz, nx;       /* physical grid */
    int W;            /* sponge width in points */
    int nt;           /* number of time samples */
    int nh;           /* number of extension points (odd): subsurface offsets, or time lags */
    double dz, dx, dt;
    int lag;          /* 0: subsurface-offset extension; > 0: time-lag extension, lags spaced lag*dt */
    int fs;           /* 1: free surface (pressure release) at the top physical row instead of a sponge */
} og_grid;

/* ------------------------------------------------------------------ grid */

int og_pad(const og_grid *g) { return g->W + 4; }
int og_NZ(const og_grid *g) { return g->nz + 2 * (g->W + 4); }
int og_NX(const og_grid *g) { return g->nx + 2 * (g->W + 4); }

static int is_active(const og_grid *g, int IZ, int IX)
{
    return IZ >= 4 && IZ < og_NZ(g) - 4 && IX >= 4 && IX < og_NX(g) - 4;
}

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* points outside the physical region along one axis (0 inside) */
static int outside(int I, int o, int n)
{
    if (I < o) return o - I;
    if (I > o + n - 1) return I - (o + n - 1);
    return 0;
}

static double taper1(int k, int W)
{
    if (k == 0 || W == 0) return 1.0;
    double a = 0.3 * (double)k / (double)W;
    return exp(-a * a);
}

/*
 * Model preparation on the padded grid.
 *   c[NZ][NX]   = v^2 dt^2 at active points (v edge-replicated), 0 elsewhere
 *   gam[NZ][NX] = sponge factor at active points, 0 elsewhere
 *   b[nz][nx]   = 2 / v^3 (physical grid; d(v^2 dt^2)/dv = c * b * v)
 */
void og_prep(const og_grid *g, const double *v, double *c, double *gam, double *b)
{
    int NZ = og_NZ(g), NX = og_NX(g), o = og_pad(g);
    for (int IZ = 0; IZ < NZ; IZ++)
        for (int IX = 0; IX < NX; IX++) {
            size_t p = (size_t)IZ * NX + IX;
            if (!is_active(g, IZ, IX) || (g->fs && IZ < o - 4)) { c[p] = 0.0; gam[p] = 0.0; continue; }
            int iz = clampi(IZ - o, 0, g->nz - 1), ix = clampi(IX - o, 0, g->nx - 1);
            double vv = v[(size_t)iz * g->nx + ix];
            c[p] = vv * vv * g->dt * g->dt;
            /* with a free surface there is no sponge on top (the mirror rows are overwritten by M) */
            double gz = (g->fs && IZ < o) ? 1.0 : taper1(outside(IZ, o, g->nz), g->W);
            gam[p] = gz * taper1(outside(IX, o, g->nx), g->W);
        }
    if (b)
        for (size_t i = 0; i < (size_t)g->nz * g->nx; i++) b[i] = 2.0 / (v[i] * v[i] * v[i]);
}

/* ------------------------------------------------------------- Laplacian */

static const double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* out = L q at active points, 0 elsewhere (L is symmetric on active fields) */
void og_lap(const og_grid *g, const double *q, double *out)
{
    int NZ = og_NZ(g), NX = og_NX(g);
    double idx2 = 1.0 / (g->dx * g->dx), idz2 = 1.0 / (g->dz * g->dz);
    for (int IZ = 0; IZ < NZ; IZ++)
        for (int IX = 0; IX < NX; IX++) {
            size_t p = (size_t)IZ * NX + IX;
            if (!is_active(g, IZ, IX)) { out[p] = 0.0; continue; }
            double sx = A8[0] * q[p], sz = A8[0] * q[p];
            for (int k = 1; k <= 4; k++) {
                sx += A8[k] * (q[p - k] + q[p + k]);
                sz += A8[k] * (q[p - (size_t)k * NX] + q[p + (size_t)k * NX]);
            }
            out[p] = sx * idx2 + sz * idz2;
        }
}

/* --------------------------------------------------------------- one step */

/* qn = gam (2 qc - gam qp + c (L qc + s)) at active points, 0 elsewhere; s may be NULL */
/* free-surface projection M: q = 0 on the surface row, odd mirror on the 4 rows above */
static void fs_project(const og_grid *g, double *q)
{
    int NX = og_NX(g), o = og_pad(g);
    for (int IX = 0; IX < NX; IX++) {
        q[(size_t)o * NX + IX] = 0.0;
        for (int k = 1; k <= 4; k++) q[(size_t)(o - k) * NX + IX] = -q[(size_t)(o + k) * NX + IX];
    }
}

/* its transpose M^T, in place on an adjoint field */
static void fs_project_T(const og_grid *g, double *a)
{
    int NX = og_NX(g), o = og_pad(g);
    for (int IX = 0; IX < NX; IX++) {
        for (int k = 1; k <= 4; k++) {
            a[(size_t)(o + k) * NX + IX] -= a[(size_t)(o - k) * NX + IX];
            a[(size_t)(o - k) * NX + IX] = 0.0;
        }
        a[(size_t)o * NX + IX] = 0.0;
    }
}

void og_step(const og_grid *g, const double *c, const double *gam, const double *qc,
             const double *qp, const double *s, double *qn)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    double *lq = (double *)malloc(P * sizeof(double));
    og_lap(g, qc, lq);
    for (size_t p = 0; p < P; p++) {
        double src = s ? s[p] : 0.0;
        qn[p] = gam[p] * (2.0 * qc[p] - gam[p] * qp[p] + c[p] * (lq[p] + src));
    }
    if (g->fs) fs_project(g, qn);
    free(lq);
}

/*
 * Literal transpose of one step, (qc, qp, s) -> qn:
 *   qc* = 2 gam qn* + L (c gam qn*),  qp* = -gam^2 qn*,  s* = c gam qn*
 * Any output pointer may be NULL.
 */
void og_step_T(const og_grid *g, const double *c, const double *gam, const double *qn_s_in,
               double *qc_s, double *qp_s, double *s_s)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    double *t = (double *)malloc(P * sizeof(double));
    double *lt = (double *)malloc(P * sizeof(double));
    double *pr = NULL;
    const double *qn_s = qn_s_in;
    if (g->fs) {   /* the step's output passes through M: its adjoint through M^T first */
        pr = (double *)malloc(P * sizeof(double));
        memcpy(pr, qn_s_in, P * sizeof(double));
        fs_project_T(g, pr);
        qn_s = pr;
    }
    for (size_t p = 0; p < P; p++) t[p] = c[p] * gam[p] * qn_s[p];
    og_lap(g, t, lt);
    for (size_t p = 0; p < P; p++) {
        if (qc_s) qc_s[p] = 2.0 * gam[p] * qn_s[p] + lt[p];
        if (qp_s) qp_s[p] = -gam[p] * gam[p] * qn_s[p];
        if (s_s) s_s[p] = t[p];
    }
    free(t);
    free(lt);
    free(pr);
}

/* ------------------------------------------------- dense time propagation */

/*
 * Forward propagation of a dense source sequence.
 *   s_seq[nt-1][P] (s^0..s^{nt-2}) -> q_seq[nt][P] (q^0..q^{nt-1}), q^{-1}=q^0=0.
 */
void og_prop(const og_grid *g, const double *c, const double *gam, const double *s_seq,
             double *q_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    double *zero = (double *)calloc(P, sizeof(double));
    memset(q_seq, 0, P * sizeof(double));
    for (int n = 0; n + 1 < g->nt; n++) {
        const double *qc = q_seq + (size_t)n * P;
        const double *qp = n > 0 ? q_seq + (size_t)(n - 1) * P : zero;
        og_step(g, c, gam, qc, qp, s_seq + (size_t)n * P, q_seq + (size_t)(n + 1) * P);
    }
    free(zero);
}

/*
 * Transpose of og_prop: a_seq[nt][P] (adjoint of q^0..q^{nt-1}) -> s*_seq[nt-1][P].
 * Adjoint recursion, backward in time, with lambda^{nt} = lambda^{nt+1} = 0:
 *   lambda^n = qc*(lambda^{n+1}) + qp*(lambda^{n+2}) + a^n,   n = nt-1 .. 1
 *   s*^n     = c gam lambda^{n+1},                            n = 0 .. nt-2
 * (q^0 is fixed at zero, so lambda^0 is not needed.)
 */
void og_prop_T(const og_grid *g, const double *c, const double *gam, const double *a_seq,
               double *ss_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    int nt = g->nt;
    double *l1 = (double *)calloc(P, sizeof(double)); /* lambda^{n+1} */
    double *l2 = (double *)calloc(P, sizeof(double)); /* lambda^{n+2} */
    double *l0 = (double *)calloc(P, sizeof(double));
    double *tc = (double *)malloc(P * sizeof(double));
    double *tp = (double *)malloc(P * sizeof(double));
    for (int n = nt - 1; n >= 1; n--) {
        og_step_T(g, c, gam, l1, tc, NULL, NULL);  /* from step n   : q^n -> q^{n+1} */
        og_step_T(g, c, gam, l2, NULL, tp, NULL);  /* from step n+1 : q^n -> q^{n+2} */
        const double *a = a_seq + (size_t)n * P;
        for (size_t p = 0; p < P; p++) l0[p] = tc[p] + tp[p] + a[p];
        /* s*^{n-1} = c gam lambda^n */
        og_step_T(g, c, gam, l0, NULL, NULL, ss_seq + (size_t)(n - 1) * P);
        double *t = l2; l2 = l1; l1 = l0; l0 = t;
    }
    free(l0); free(l1); free(l2); free(tc); free(tp);
}

/* ------------------------------------------------------ time derivative */

/* D^n = (q^{n+1} - 2 q^n + q^{n-1}) / dt^2, n = 0..nt-2, q^{-1} = 0 */
void og_d2t(const og_grid *g, const double *q_seq, double *D_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    double idt2 = 1.0 / (g->dt * g->dt);
    for (int n = 0; n + 1 < g->nt; n++)
        for (size_t p = 0; p < P; p++) {
            double qm = n > 0 ? q_seq[(size_t)(n - 1) * P + p] : 0.0;
            D_seq[(size_t)n * P + p] =
                (q_seq[(size_t)(n + 1) * P + p] - 2.0 * q_seq[(size_t)n * P + p] + qm) * idt2;
        }
}

/* transpose: z[nt-1][P] -> a[nt][P], a^m = (z^{m-1} - 2 z^m + z^{m+1}) / dt^2 */
void og_d2t_T(const og_grid *g, const double *z_seq, double *a_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    int nt = g->nt;
    double idt2 = 1.0 / (g->dt * g->dt);
    for (int m = 0; m < nt; m++)
        for (size_t p = 0; p < P; p++) {
            double zm1 = (m - 1 >= 0 && m - 1 <= nt - 2) ? z_seq[(size_t)(m - 1) * P + p] : 0.0;
            double z0 = (m <= nt - 2) ? z_seq[(size_t)m * P + p] : 0.0;
            double zp1 = (m + 1 <= nt - 2) ? z_seq[(size_t)(m + 1) * P + p] : 0.0;
            a_seq[(size_t)m * P + p] = (zm1 - 2.0 * z0 + zp1) * idt2;
        }
}

/* -------------------------------------------- record / inject (R, R^T) */

/* d[r] = q(rec_r); receivers in physical indices */
void og_record(const og_grid *g, const double *q, int nrec, const int *rec_iz,
               const int *rec_ix, double *d)
{
    int NX = og_NX(g), o = og_pad(g);
    for (int r = 0; r < nrec; r++) d[r] = q[(size_t)(rec_iz[r] + o) * NX + rec_ix[r] + o];
}

/* q(rec_r) += d[r] */
void og_inject(const og_grid *g, const double *d, int nrec, const int *rec_iz,
               const int *rec_ix, double *q)
{
    int NX = og_NX(g), o = og_pad(g);
    for (int r = 0; r < nrec; r++) q[(size_t)(rec_iz[r] + o) * NX + rec_ix[r] + o] += d[r];
}

/* ----------------------------------------------- extended scatter E(W, D) */

/*
 * e(y) = sum_h W(y-h, h) D(y-2h); W[nh][nz][nx] on the physical grid, e and D
 * padded.  Written as a loop over scatter points x (physical) and offsets h:
 * the point x couples D at x-h to e at x+h.  Terms with x-h or x+h outside
 * the active region are dropped.  Overwrites e.
 */
void og_scatter(const og_grid *g, const double *Wt, const double *D, double *e)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t P = (size_t)og_NZ(g) * NX, PP = (size_t)g->nz * g->nx;
    memset(e, 0, P * sizeof(double));
    for (int ih = 0; ih < g->nh; ih++) {
        int h = ih - hm;
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                int IZ = iz + o, IX = ix + o;
                if (!is_active(g, IZ, IX - h) || !is_active(g, IZ, IX + h)) continue;
                e[(size_t)IZ * NX + IX + h] +=
                    Wt[ih * PP + (size_t)iz * g->nx + ix] * D[(size_t)IZ * NX + IX - h];
            }
    }
}

/* transpose w.r.t. D:  z(u) = sum_h W(u+h, h) e*(u+2h).  Overwrites z. */
void og_scatter_TD(const og_grid *g, const double *Wt, const double *es, double *z)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t P = (size_t)og_NZ(g) * NX, PP = (size_t)g->nz * g->nx;
    memset(z, 0, P * sizeof(double));
    for (int ih = 0; ih < g->nh; ih++) {
        int h = ih - hm;
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                int IZ = iz + o, IX = ix + o;
                if (!is_active(g, IZ, IX - h) || !is_active(g, IZ, IX + h)) continue;
                z[(size_t)IZ * NX + IX - h] +=
                    Wt[ih * PP + (size_t)iz * g->nx + ix] * es[(size_t)IZ * NX + IX + h];
            }
    }
}

/* transpose w.r.t. W:  W*(x, h) += D(x-h) e*(x+h)  (accumulates into Ws) */
void og_scatter_TW_acc(const og_grid *g, const double *D, const double *es, double *Ws)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t PP = (size_t)g->nz * g->nx;
    for (int ih = 0; ih < g->nh; ih++) {
        int h = ih - hm;
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                int IZ = iz + o, IX = ix + o;
                if (!is_active(g, IZ, IX - h) || !is_active(g, IZ, IX + h)) continue;
                Ws[ih * PP + (size_t)iz * g->nx + ix] +=
                    D[(size_t)IZ * NX + IX - h] * es[(size_t)IZ * NX + IX + h];
            }
    }
}

/* zero-embedding of a physical field into the padded grid */
static void embed(const og_grid *g, const double *a, double *A)
{
    int NX = og_NX(g), o = og_pad(g);
    memset(A, 0, (size_t)og_NZ(g) * NX * sizeof(double));
    for (int iz = 0; iz < g->nz; iz++)
        for (int ix = 0; ix < g->nx; ix++)
            A[(size_t)(iz + o) * NX + ix + o] = a[(size_t)iz * g->nx + ix];
}

/* ================================================================ shots ==
 * A shot: one point source at physical (src_iz, src_ix) with wavelet w[nt],
 * receivers at physical (rec_iz[r], rec_ix[r]); data d[nt][nrec].
 */
typedef struct {
    int src_iz, src_ix;
    const double *w;
    int nrec;
    const int *rec_iz, *rec_ix;
} og_shot;

/* dense point-source sequence s^n = w[n]/(dx dz) at the source, n = 0..nt-2 */
static double *point_source_seq(const og_grid *g, const og_shot *sh)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    int NX = og_NX(g), o = og_pad(g);
    double *s = (double *)calloc((size_t)(g->nt - 1) * P, sizeof(double));
    size_t ps = (size_t)(sh->src_iz + o) * NX + sh->src_ix + o;
    for (int n = 0; n + 1 < g->nt; n++) s[(size_t)n * P + ps] = sh->w[n] / (g->dx * g->dz);
    return s;
}

static void record_seq(const og_grid *g, const og_shot *sh, const double *q_seq, double *d)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    for (int n = 0; n < g->nt; n++)
        og_record(g, q_seq + (size_t)n * P, sh->nrec, sh->rec_iz, sh->rec_ix, d + (size_t)n * sh->nrec);
}

static double *inject_seq(const og_grid *g, const og_shot *sh, const double *d)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    double *a = (double *)calloc((size_t)g->nt * P, sizeof(double));
    for (int n = 0; n < g->nt; n++)
        og_inject(g, d + (size_t)n * sh->nrec, sh->nrec, sh->rec_iz, sh->rec_ix, a + (size_t)n * P);
    return a;
}

typedef struct {
    size_t P, PP;
    double *c, *gam, *b, *bpad;
} model_t;

static void model_init(const og_grid *g, const double *v, model_t *m)
{
    m->P = (size_t)og_NZ(g) * og_NX(g);
    m->PP = (size_t)g->nz * g->nx;
    m->c = (double *)malloc(m->P * sizeof(double));
    m->gam = (double *)malloc(m->P * sizeof(double));
    m->b = (double *)malloc(m->PP * sizeof(double));
    m->bpad = (double *)malloc(m->P * sizeof(double));
    og_prep(g, v, m->c, m->gam, m->b);
    embed(g, m->b, m->bpad);
}

static void model_free(model_t *m) { free(m->c); free(m->gam); free(m->b); free(m->bpad); }

/* q0 history and its D2t history for one shot (background wavefield) */
static void background(const og_grid *g, const model_t *m, const og_shot *sh, double **q0, double **D0)
{
    size_t P = m->P;
    double *s = point_source_seq(g, sh);
    *q0 = (double *)malloc((size_t)g->nt * P * sizeof(double));
    og_prop(g, m->c, m->gam, s, *q0);
    free(s);
    if (D0) {
        *D0 = (double *)malloc((size_t)(g->nt - 1) * P * sizeof(double));
        og_d2t(g, *q0, *D0);
    }
}

/* W = b * p~ on the physical grid, per offset */
static double *ext_weights(const og_grid *g, const model_t *m, const double *pt)
{
    double *Wt = (double *)malloc((size_t)g->nh * m->PP * sizeof(double));
    for (int ih = 0; ih < g->nh; ih++)
        for (size_t i = 0; i < m->PP; i++) Wt[ih * m->PP + i] = m->b[i] * pt[ih * m->PP + i];
    return Wt;
}

/*
 * f(m): Eq. 1 nonlinear forward, d[nt][nrec].  Written as the plain time loop
 * of the recursion (three time levels), recording q^n before stepping.
 */
void og_forward(const og_grid *g, const double *v, const og_shot *sh, double *d)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P;
    int NX = og_NX(g), o = og_pad(g);
    double *qp = (double *)calloc(P, sizeof(double)), *qc = (double *)calloc(P, sizeof(double));
    double *qn = (double *)calloc(P, sizeof(double)), *s = (double *)calloc(P, sizeof(double));
    size_t ps = (size_t)(sh->src_iz + o) * NX + sh->src_ix + o;
    for (int n = 0; n < g->nt; n++) {
        og_record(g, qc, sh->nrec, sh->rec_iz, sh->rec_ix, d + (size_t)n * sh->nrec);
        if (n + 1 == g->nt) break;
        s[ps] = sh->w[n] / (g->dx * g->dz);
        og_step(g, m.c, m.gam, qc, qp, s, qn);
        double *t = qp; qp = qc; qc = qn; qn = t;
    }
    free(qp); free(qc); free(qn); free(s); model_free(&m);
}

/* B(m) dv: Born, secondary source b dv D2t q0 (Eq. 8 operator) */
void og_born(const og_grid *g, const double *v, const og_shot *sh, const double *dv, double *d)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P;
    double *q0, *D0; background(g, &m, sh, &q0, &D0);
    double *dvp = (double *)malloc(P * sizeof(double)); embed(g, dv, dvp);
    double *s = (double *)malloc((size_t)(g->nt - 1) * P * sizeof(double));
    for (int n = 0; n + 1 < g->nt; n++)
        for (size_t p = 0; p < P; p++) s[(size_t)n * P + p] = m.bpad[p] * dvp[p] * D0[(size_t)n * P + p];
    double *dq = (double *)malloc((size_t)g->nt * P * sizeof(double));
    og_prop(g, m.c, m.gam, s, dq);
    record_seq(g, sh, dq, d);
    free(q0); free(D0); free(dvp); free(s); free(dq); model_free(&m);
}

/* B*(m) d: adjoint Born, g[nz][nx] = b sum_n D2t q0^n * s*^n (overwrites) */
void og_born_adj(const og_grid *g, const double *v, const og_shot *sh, const double *d, double *gout)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P;
    int NX = og_NX(g), o = og_pad(g);
    double *q0, *D0; background(g, &m, sh, &q0, &D0);
    double *a = inject_seq(g, sh, d);
    double *ss = (double *)malloc((size_t)(g->nt - 1) * P * sizeof(double));
    og_prop_T(g, m.c, m.gam, a, ss);
    for (int iz = 0; iz < g->nz; iz++)
        for (int ix = 0; ix < g->nx; ix++) {
            size_t p = (size_t)(iz + o) * NX + ix + o;
            double acc = 0.0;
            for (int n = 0; n + 1 < g->nt; n++) acc += D0[(size_t)n * P + p] * ss[(size_t)n * P + p];
            gout[(size_t)iz * g->nx + ix] = m.b[(size_t)iz * g->nx + ix] * acc;
        }
    free(q0); free(D0); free(a); free(ss); model_free(&m);
}

/* B~(m) p~: extended Born (subsurface offsets) */
/* Transpose of og_scatter_tlag w.r.t. D: z^m(x) = sum_i W(x, i) es^{m + 2 s_i}(x).  Overwrites z. */
void og_scatter_tlag_TD(const og_grid *g, const double *Wt, const double *es_seq, int m, double *z)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t P = (size_t)og_NZ(g) * NX, PP = (size_t)g->nz * g->nx;
    memset(z, 0, P * sizeof(double));
    for (int i = 0; i < g->nh; i++) {
        int n = m + 2 * (i - hm) * g->lag;
        if (n < 0 || n > g->nt - 2) continue;
        const double *es = es_seq + (size_t)n * P;
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                size_t at = (size_t)(iz + o) * NX + ix + o;
                z[at] += Wt[i * PP + (size_t)iz * g->nx + ix] * es[at];
            }
    }
}

/* Transpose of og_scatter_tlag w.r.t. W, accumulated: Ws(x, i) += sum_n D^{n - 2 s_i}(x) es^n(x) */
void og_scatter_tlag_TW_acc(const og_grid *g, const double *D_seq, const double *es_seq, double *Ws)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t P = (size_t)og_NZ(g) * NX, PP = (size_t)g->nz * g->nx;
    for (int i = 0; i < g->nh; i++)
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                size_t at = (size_t)(iz + o) * NX + ix + o;
                double acc = 0.0;
                for (int n = 0; n + 1 < g->nt; n++) {
                    int mm = n - 2 * (i - hm) * g->lag;
                    if (mm < 0 || mm > g->nt - 2) continue;
                    acc += D_seq[(size_t)mm * P + at] * es_seq[(size_t)n * P + at];
                }
                Ws[i * PP + (size_t)iz * g->nx + ix] += acc;
            }
}

void og_scatter_tlag(const og_grid *g, const double *Wt, const double *D_seq, int n, double *e);

/* The extension over whole sequences (steps 0..nt-2): subsurface offsets (lag = 0) or time lags */
static void ext_scatter_seq(const og_grid *g, const double *Wt, const double *D_seq, double *e_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    for (int n = 0; n + 1 < g->nt; n++) {
        if (g->lag > 0) og_scatter_tlag(g, Wt, D_seq, n, e_seq + (size_t)n * P);
        else og_scatter(g, Wt, D_seq + (size_t)n * P, e_seq + (size_t)n * P);
    }
}
static void ext_scatter_TD_seq(const og_grid *g, const double *Wt, const double *es_seq, double *z_seq)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    for (int n = 0; n + 1 < g->nt; n++) {
        if (g->lag > 0) og_scatter_tlag_TD(g, Wt, es_seq, n, z_seq + (size_t)n * P);
        else og_scatter_TD(g, Wt, es_seq + (size_t)n * P, z_seq + (size_t)n * P);
    }
}
static void ext_scatter_TW_seq(const og_grid *g, const double *D_seq, const double *es_seq, double *Ws)
{
    size_t P = (size_t)og_NZ(g) * og_NX(g);
    if (g->lag > 0) {
        og_scatter_tlag_TW_acc(g, D_seq, es_seq, Ws);
        return;
    }
    for (int n = 0; n + 1 < g->nt; n++) og_scatter_TW_acc(g, D_seq + (size_t)n * P, es_seq + (size_t)n * P, Ws);
}

/* B~(m) p~ (either extension): scatter every step, propagate, record */
void og_born_ext(const og_grid *g, const double *v, const og_shot *sh, const double *pt, double *d)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P;
    double *q0, *D0; background(g, &m, sh, &q0, &D0);
    double *Wt = ext_weights(g, &m, pt);
    double *s = (double *)malloc((size_t)(g->nt - 1) * P * sizeof(double));
    ext_scatter_seq(g, Wt, D0, s);
    double *dq = (double *)malloc((size_t)g->nt * P * sizeof(double));
    og_prop(g, m.c, m.gam, s, dq);
    record_seq(g, sh, dq, d);
    free(q0); free(D0); free(Wt); free(s); free(dq); model_free(&m);
}

/* B~*(m) d: extended imaging condition, pt[nh][nz][nx] = b(x) sum_n D0^n(x-h) s*^n(x+h) (offsets) or
 * b(x) sum_n D0^{n - 2 s_i}(x) s*^n(x) (time lags) */
void og_born_ext_adj(const og_grid *g, const double *v, const og_shot *sh, const double *d, double *pt)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P, PP = m.PP;
    double *q0, *D0; background(g, &m, sh, &q0, &D0);
    double *a = inject_seq(g, sh, d);
    double *ss = (double *)malloc((size_t)(g->nt - 1) * P * sizeof(double));
    og_prop_T(g, m.c, m.gam, a, ss);
    double *Ws = (double *)calloc((size_t)g->nh * PP, sizeof(double));
    ext_scatter_TW_seq(g, D0, ss, Ws);
    for (int ih = 0; ih < g->nh; ih++)
        for (size_t i = 0; i < PP; i++) pt[ih * PP + i] = m.b[i] * Ws[ih * PP + i];
    free(q0); free(D0); free(a); free(ss); free(Ws); model_free(&m);
}

/*
 * Time-lag extension (Theory section: B~ is Born modelling extended with time
 * lags or with horizontal subsurface offsets, Eq. 1).  Symmetric convention:
 * lag tau_i = s_i dt, s_i = (i - hm) lag, couples the source wavefield at
 * t - tau with the receiver side at t + tau, so the secondary source of step n
 * reads the background's D2t 2 s_i steps earlier:
 *   e^n(x) = sum_i W(x, i) D^{n - 2 s_i}(x),   W = b p~,   D^m = 0 unless 0 <= m <= nt-2.
 * Overwrites e (physical points only carry weights).
 */
void og_scatter_tlag(const og_grid *g, const double *Wt, const double *D_seq, int n, double *e)
{
    int NX = og_NX(g), o = og_pad(g), hm = (g->nh - 1) / 2;
    size_t P = (size_t)og_NZ(g) * NX, PP = (size_t)g->nz * g->nx;
    memset(e, 0, P * sizeof(double));
    for (int i = 0; i < g->nh; i++) {
        int m = n - 2 * (i - hm) * g->lag;
        if (m < 0 || m > g->nt - 2) continue;
        const double *D = D_seq + (size_t)m * P;
        for (int iz = 0; iz < g->nz; iz++)
            for (int ix = 0; ix < g->nx; ix++) {
                size_t at = (size_t)(iz + o) * NX + ix + o;
                e[at] += Wt[i * PP + (size_t)iz * g->nx + ix] * D[at];
            }
    }
}

/*
 * T(m, p~) dv: derivative of m -> B~(m) p~ along dv (Eq. 9 operator).  Three
 * secondary sources drive one more propagation:
 *   (i)   b dv D2t dqs           dqs = extended Born wavefield of p~
 *   (ii)  E(W', D0), W' = (-3 dv / v) b p~     (from db/dv = -3 b / v)
 *   (iii) E(W, D2t dq0)          dq0 = Born wavefield of dv
 */
void og_tomo(const og_grid *g, const double *v, const og_shot *sh, const double *pt,
             const double *dv, double *d)
{
    model_t m; model_init(g, v, &m);
    size_t P = m.P, PP = m.PP, SP = (size_t)(g->nt - 1) * P, QP = (size_t)g->nt * P;
    double *q0, *D0; background(g, &m, sh, &q0, &D0);
    double *Wt = ext_weights(g, &m, pt);
    double *W2 = (double *)malloc((size_t)g->nh * PP * sizeof(double));
    for (int ih = 0; ih < g->nh; ih++)
        for (size_t i = 0; i < PP; i++) W2[ih * PP + i] = -3.0 * dv[i] / v[i] * Wt[ih * PP + i];
    double *dvp = (double *)malloc(P * sizeof(double)); embed(g, dv, dvp);
    double *s = (double *)malloc(SP * sizeof(double));
    double *tmp = (double *)malloc(P * sizeof(double));
    double *dq0 = (double *)malloc(QP * sizeof(double)), *Dq0 = (double *)malloc(SP * sizeof(double));
    double *dqs = (double *)malloc(QP * sizeof(double)), *Dqs = (double *)malloc(SP * sizeof(double));
    /* dq0: Born wavefield of dv */
    for (int n = 0; n + 1 < g->nt; n++)
        for (size_t p = 0; p < P; p++) s[(size_t)n * P + p] = m.bpad[p] * dvp[p] * D0[(size_t)n * P + p];
    og_prop(g, m.c, m.gam, s, dq0);
    og_d2t(g, dq0, Dq0);
    /* dqs: extended Born wavefield of p~ */
    ext_scatter_seq(g, Wt, D0, s);
    og_prop(g, m.c, m.gam, s, dqs);
    og_d2t(g, dqs, Dqs);
    /* the three secondary sources of T dv */
    double *e2 = (double *)malloc(SP * sizeof(double)), *e3 = (double *)malloc(SP * sizeof(double));
    ext_scatter_seq(g, W2, D0, e2);
    ext_scatter_seq(g, Wt, Dq0, e3);
    for (int n = 0; n + 1 < g->nt; n++) {
        double *sn = s + (size_t)n * P;
        for (size_t p = 0; p < P; p++) sn[p] = m.bpad[p] * dvp[p] * Dqs[(size_t)n * P + p];
        for (size_t p = 0; p < P; p++) sn[p] += e2[(size_t)n * P + p];
        for (size_t p = 0; p < P; p++) sn[p] += e3[(size_t)n * P + p];
    }
    free(e2); free(e3);
    double *dqt = (double *)malloc(QP * sizeof(double));
    og_prop(g, m.c, m.gam, s, dqt);
    record_seq(g, sh, dqt, d);
    free(q0); free(D0); free(Wt); free(W2); free(dvp); free(s); free(tmp);
    free(dq0); free(Dq0); free(dqs); free(Dqs); free(dqt); model_free(&m);
}

/*
 * Shared backward part of T* and of the gradient.  Given the adjoint source
 * sequence a (injected residual), accumulates into gout[nz][nx]:
 *   born_term:  b sum_n D0^n s*^n                       (B* r)
 *   (i)         b sum_n D2t dqs^n s*^n
 *   (ii)        -3/v sum_h p~(x,h) [ b sum_n D0^n(x-h) s*^n(x+h) ]
 *   (iii)       b sum_n D0^n s2*^n,  s2* = prop^T( d2t^T( E_D^T(W, s*) ) )
 */
static void tomo_adj_core(const og_grid *g, const double *v, const model_t *m, const og_shot *sh,
                          const double *pt, const double *r, int born_term, double *gout)
{
    size_t P = m->P, PP = m->PP, SP = (size_t)(g->nt - 1) * P, QP = (size_t)g->nt * P;
    int NX = og_NX(g), o = og_pad(g), nt = g->nt;
    double *q0, *D0; background(g, m, sh, &q0, &D0);
    double *Wt = ext_weights(g, m, pt);
    double *s = (double *)malloc(SP * sizeof(double));
    double *dqs = (double *)malloc(QP * sizeof(double)), *Dqs = (double *)malloc(SP * sizeof(double));
    ext_scatter_seq(g, Wt, D0, s);
    og_prop(g, m->c, m->gam, s, dqs);
    og_d2t(g, dqs, Dqs);
    /* adjoint wavefield of the residual */
    double *a = inject_seq(g, sh, r);
    double *ss = (double *)malloc(SP * sizeof(double));
    og_prop_T(g, m->c, m->gam, a, ss);
    /* term (ii): extended image of r, contracted with p~ */
    double *Ws = (double *)calloc((size_t)g->nh * PP, sizeof(double));
    ext_scatter_TW_seq(g, D0, ss, Ws);
    /* term (iii): z^n = E_D^T(W, s*^n), then d2t^T, then prop^T */
    double *z = (double *)malloc(SP * sizeof(double));
    ext_scatter_TD_seq(g, Wt, ss, z);
    double *a2 = (double *)malloc(QP * sizeof(double));
    og_d2t_T(g, z, a2);
    double *ss2 = (double *)malloc(SP * sizeof(double));
    og_prop_T(g, m->c, m->gam, a2, ss2);
    for (int iz = 0; iz < g->nz; iz++)
        for (int ix = 0; ix < g->nx; ix++) {
            size_t p = (size_t)(iz + o) * NX + ix + o, i = (size_t)iz * g->nx + ix;
            double acc_b = 0.0, acc_i = 0.0, acc_iii = 0.0, acc_ii = 0.0;
            for (int n = 0; n + 1 < nt; n++) {
                size_t q = (size_t)n * P + p;
                acc_b += D0[q] * ss[q];
                acc_i += Dqs[q] * ss[q];
                acc_iii += D0[q] * ss2[q];
            }
            for (int ih = 0; ih < g->nh; ih++) acc_ii += pt[ih * PP + i] * m->b[i] * Ws[ih * PP + i];
            double val = m->b[i] * acc_i + (-3.0 / v[i]) * acc_ii + m->b[i] * acc_iii;
            if (born_term) val += m->b[i] * acc_b;
            gout[i] += val;
        }
    free(q0); free(D0); free(Wt); free(s); free(dqs); free(Dqs); free(a); free(ss);
    free(Ws); free(z); free(a2); free(ss2);
}

/* T*(m, p~) d -> gout[nz][nx] (overwrites) */
void og_tomo_adj(const og_grid *g, const double *v, const og_shot *sh, const double *pt,
                 const double *d, double *gout)
{
    model_t m; model_init(g, v, &m);
    memset(gout, 0, m.PP * sizeof(double));
    tomo_adj_core(g, v, &m, sh, pt, d, 0, gout);
    model_free(&m);
}

/*
 * FWIME objective at fixed p~ and its gradient for one shot (S = I):
 *   r = f(m) + B~(m) p~ - d_obs
 *   J = 1/2 ||r||^2                (the eps^2/2 ||D p~||^2 term is added once
 *                                   per model by og_dso_penalty, not per shot)
 *   g = B* r + T* r                (Eqs. 7-9)
 * r_out[nt][nrec] (may be NULL) receives the residual; gout is overwritten.
 */
double og_gradient(const og_grid *g, const double *v, const og_shot *sh, const double *pt,
                   const double *dobs, double *gout, double *r_out)
{
    model_t m; model_init(g, v, &m);
    size_t nd = (size_t)g->nt * sh->nrec;
    double *f = (double *)malloc(nd * sizeof(double));
    double *bp = (double *)malloc(nd * sizeof(double));
    double *r = (double *)malloc(nd * sizeof(double));
    og_forward(g, v, sh, f);
    og_born_ext(g, v, sh, pt, bp);
    double J = 0.0;
    for (size_t i = 0; i < nd; i++) {
        r[i] = f[i] + bp[i] - dobs[i];
        J += 0.5 * r[i] * r[i];
    }
    if (r_out) memcpy(r_out, r, nd * sizeof(double));
    memset(gout, 0, m.PP * sizeof(double));
    tomo_adj_core(g, v, &m, sh, pt, r, 1, gout);
    free(f); free(bp); free(r); model_free(&m);
    return J;
}

/*
 * eps^2/2 ||D p~||^2 with D = diag(|ih - hm| + 1): one reading of the
 * invertible, modified DSO operator named in the Theory section.
 */
double og_dso_penalty(const og_grid *g, const double *pt, double eps)
{
    int hm = (g->nh - 1) / 2;
    size_t PP = (size_t)g->nz * g->nx;
    double acc = 0.0;
    for (int ih = 0; ih < g->nh; ih++) {
        double w = fabs((double)(ih - hm)) + 1.0;
        for (size_t i = 0; i < PP; i++) {
            double t = w * pt[ih * PP + i];
            acc += t * t;
        }
    }
    return 0.5 * eps * eps * acc;
}

/* ----------------------------------------------------------- cost model */

/* Computational-aspects section, Eq. 10 and Eq. 11: C_vp and C_FWIME */
double og_cost_vp(int n_vp, double c_ext) { return 4.0 * n_vp * (1.0 + c_ext); }
double og_cost_fwime(int n_vp, double c_ext) { return 6.0 + og_cost_vp(n_vp, c_ext); }

/* ========================================================= many shots ====
 * Plain loop over shots; shots may run on several host threads (OpenMP), each
 * shot writes its own slice; summed outputs are summed in shot order.
 * w[nshot][nt], src_iz/src_ix[nshot], fixed receiver spread, d[nshot][nt][nrec].
 */
typedef enum { OP_FWD = 0, OP_BORN, OP_BORN_ADJ, OP_EXT, OP_EXT_ADJ, OP_TOMO, OP_TOMO_ADJ, OP_GRAD } op_t;

static og_shot make_shot(const og_grid *g, int s, const int *src_iz, const int *src_ix, const double *w,
                         int nrec, const int *rec_iz, const int *rec_ix)
{
    og_shot sh;
    sh.src_iz = src_iz[s]; sh.src_ix = src_ix[s];
    sh.w = w + (size_t)s * g->nt;
    sh.nrec = nrec; sh.rec_iz = rec_iz; sh.rec_ix = rec_ix;
    return sh;
}

/*
 * Runs operator `op` over nshot shots.
 *   data-space outputs (FWD, BORN, EXT, TOMO) are written per shot to out[nshot][nt][nrec]
 *   model-space outputs (BORN_ADJ, EXT_ADJ, TOMO_ADJ, GRAD) are summed over shots into out
 * in1 = dv (BORN, TOMO) or p~ (EXT, TOMO_ADJ, GRAD) or data (BORN_ADJ, EXT_ADJ, TOMO_ADJ: in2)
 * Returns J summed over shots for GRAD (without the DSO term), else 0.
 */
double og_shots(const og_grid *g, int op, const double *v, int nshot, const int *src_iz,
                const int *src_ix, const double *w, int nrec, const int *rec_iz, const int *rec_ix,
                const double *in1, const double *in2, double *out, int nthreads)
{
    size_t PP = (size_t)g->nz * g->nx, nd = (size_t)g->nt * nrec;
    size_t mlen = (op == OP_EXT_ADJ) ? (size_t)g->nh * PP : PP;
    int model_out = (op == OP_BORN_ADJ || op == OP_EXT_ADJ || op == OP_TOMO_ADJ || op == OP_GRAD);
    double *part = model_out ? (double *)calloc((size_t)nshot * mlen, sizeof(double)) : NULL;
    double *Js = (double *)calloc((size_t)nshot, sizeof(double));
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int s = 0; s < nshot; s++) {
        og_shot sh = make_shot(g, s, src_iz, src_ix, w, nrec, rec_iz, rec_ix);
        double *o = model_out ? part + (size_t)s * mlen : out + (size_t)s * nd;
        const double *ds = in2 ? in2 + (size_t)s * nd : NULL;
        switch (op) {
        case OP_FWD: og_forward(g, v, &sh, o); break;
        case OP_BORN: og_born(g, v, &sh, in1, o); break;
        case OP_BORN_ADJ: og_born_adj(g, v, &sh, ds, o); break;
        case OP_EXT: og_born_ext(g, v, &sh, in1, o); break;
        case OP_EXT_ADJ: og_born_ext_adj(g, v, &sh, ds, o); break;
        case OP_TOMO: og_tomo(g, v, &sh, in1, in2 ? in2 : NULL, o); break;
        case OP_TOMO_ADJ: og_tomo_adj(g, v, &sh, in1, ds, o); break;
        case OP_GRAD: Js[s] = og_gradient(g, v, &sh, in1, ds, o, NULL); break;
        }
    }
    double J = 0.0;
    if (model_out) {
        memset(out, 0, mlen * sizeof(double));
        for (int s = 0; s < nshot; s++)
            for (size_t i = 0; i < mlen; i++) out[i] += part[(size_t)s * mlen + i];
    }
    for (int s = 0; s < nshot; s++) J += Js[s];
    free(part); free(Js);
    return J;
}
