/*
 * ssx_oracle.c -- FP64 CPU oracle: one leapfrog step of the staggered-grid
 * acoustic system and its exact transpose, plus whole-sweep drivers.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may load this file's
 * library: only tests, the smoke check and the benchmark's CPU-baseline and
 * reference legs use it. It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (W. W. Symes, "Efficient Computation of Extended Surface
 * Sources", arXiv 2203.16573):
 *   - the acoustic system of eqn:awepm, (1/kappa) p_t = -div v + h delta(z-z_s),
 *     rho v_t = -grad p + f e_z delta(z-z_s), discretised as in the section
 *     "Synthetic models and simulation": staggered grid, order 2 in time and 2k
 *     in space, linear-interpolation sampling and adjoint-interpolation
 *     injection; an absorbing sponge replaces the paper's PML;
 *   - the exact discrete transpose of that sweep (Appendix A: the adjoint
 *     state / reverse-time computation, here written out by hand).
 *
 * Discrete conventions (binding for every consumer of the oracle):
 *   p(i,k) at (i h, k h); vx(j,k) at ((j+1/2) h, k h), j in [0, NX-2];
 *   vz(i,k) at (i h, (k+1/2) h), k in [0, NZ-2]; fields are zero outside.
 *   Step n: v^{n+1/2} = A_v v^{n-1/2} - B_v dt/(rho h) D+ p^n  (+ f[n] injection)
 *           p^{n+1}   = A_p p^n - B_p kappa dt/h D- v^{n+1/2}  (+ h[n] injection)
 *           samples:  P p^{n+1},  P vz^{n+1/2}
 *   with A = (1 - s)/(1 + s), B = 1/(1 + s), s = (sigma_x + sigma_z) dt/2
 *   evaluated at each field's own position.
 *   D+ u (j+1/2) = sum_m c_m (u[j+m] - u[j-m+1]);
 *   D- w (i)     = sum_m c_m (w[i+m-1] - w[i-m]).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int NX, NZ;          /* padded grid (p points) */
    int R;               /* half-order k: 2k-th order differences */
    double c[8];         /* staggered difference weights c_1..c_k */
    double dt, h, rho;
    const double *kappa; /* [NZ*NX] bulk modulus at p points */
    const double *sx_i;  /* [NX] sponge sigma at x = i h      */
    const double *sx_h;  /* [NX] sponge sigma at x = (i+1/2) h */
    const double *sz_i;  /* [NZ] sponge sigma at z = k h      */
    const double *sz_h;  /* [NZ] sponge sigma at z = (k+1/2) h */
} og_grid;

/* A line of injection/sampling points: columns i0..i0+n-1 at one depth.
 * Pressure rows kp, kp+1 with weights wp0, wp1 (linear interpolation in z on
 * the integer rows); vz rows kv, kv+1 with weights wv0, wv1 (on the half rows).
 * scale multiplies injected values (1 for a line density, 1/h for a point). */
typedef struct {
    int i0, n;
    int kp;
    double wp0, wp1;
    int kv;
    double wv0, wv1;
    double scale;
} og_line;

static inline double P(const og_grid *g, const double *p, int k, int i) {
    if (i < 0 || i >= g->NX || k < 0 || k >= g->NZ) return 0.0;
    return p[(size_t)k * g->NX + i];
}
static inline double VX(const og_grid *g, const double *vx, int k, int j) {
    if (j < 0 || j >= g->NX - 1 || k < 0 || k >= g->NZ) return 0.0;
    return vx[(size_t)k * g->NX + j];
}
static inline double VZ(const og_grid *g, const double *vz, int k, int i) {
    if (i < 0 || i >= g->NX || k < 0 || k >= g->NZ - 1) return 0.0;
    return vz[(size_t)k * g->NX + i];
}
/* damping factors for a point whose total sigma is sig */
static inline double damp_a(const og_grid *g, double sig) {
    double s = 0.5 * sig * g->dt;
    return (1.0 - s) / (1.0 + s);
}
static inline double damp_b(const og_grid *g, double sig) {
    return 1.0 / (1.0 + 0.5 * sig * g->dt);
}
/* coefficient of the v update (without the D+ p factor) */
static inline double cvx(const og_grid *g, int k, int j) {
    return damp_b(g, g->sx_h[j] + g->sz_i[k]) * g->dt / (g->rho * g->h);
}
static inline double cvz(const og_grid *g, int k, int i) {
    return damp_b(g, g->sx_i[i] + g->sz_h[k]) * g->dt / (g->rho * g->h);
}
static inline double cp(const og_grid *g, int k, int i) {
    return damp_b(g, g->sx_i[i] + g->sz_i[k]) * g->kappa[(size_t)k * g->NX + i] * g->dt / g->h;
}

/* One forward step n (in place): p^n, v^{n-1/2} -> p^{n+1}, v^{n+1/2}.
 * hrow/frow: pressure / velocity source samples of step n on `src` (or NULL).
 * prow/vrow: receive P p^{n+1} / P vz^{n+1/2} on `rec` (or NULL). */
void og_step_fwd(const og_grid *g, double *p, double *vx, double *vz,
                 const og_line *src, const double *hrow, const double *frow,
                 const og_line *rec, double *prow, double *vrow)
{
    const int NX = g->NX, NZ = g->NZ, R = g->R;
    /* velocity half step: rho v_t = -grad p */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++) {
        for (int j = 0; j < NX - 1; j++) {
            double d = 0.0;
            for (int m = 1; m <= R; m++)
                d += g->c[m - 1] * (P(g, p, k, j + m) - P(g, p, k, j - m + 1));
            size_t o = (size_t)k * NX + j;
            vx[o] = damp_a(g, g->sx_h[j] + g->sz_i[k]) * vx[o] - cvx(g, k, j) * d;
        }
        if (k < NZ - 1) {
            for (int i = 0; i < NX; i++) {
                double d = 0.0;
                for (int m = 1; m <= R; m++)
                    d += g->c[m - 1] * (P(g, p, k + m, i) - P(g, p, k - m + 1, i));
                size_t o = (size_t)k * NX + i;
                vz[o] = damp_a(g, g->sx_i[i] + g->sz_h[k]) * vz[o] - cvz(g, k, i) * d;
            }
        }
    }
    /* vertical load f e_z delta(z - z_s), adjoint linear interpolation */
    if (frow) {
        for (int j = 0; j < src->n; j++) {
            int i = src->i0 + j;
            double s = src->scale * frow[j];
            vz[(size_t)src->kv * NX + i] += cvz(g, src->kv, i) * src->wv0 * s;
            if (src->wv1 != 0.0)
                vz[(size_t)(src->kv + 1) * NX + i] += cvz(g, src->kv + 1, i) * src->wv1 * s;
        }
    }
    /* pressure half step: (1/kappa) p_t = -div v */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++) {
        for (int i = 0; i < NX; i++) {
            double d = 0.0;
            for (int m = 1; m <= R; m++) {
                d += g->c[m - 1] * (VX(g, vx, k, i + m - 1) - VX(g, vx, k, i - m));
                d += g->c[m - 1] * (VZ(g, vz, k + m - 1, i) - VZ(g, vz, k - m, i));
            }
            size_t o = (size_t)k * NX + i;
            p[o] = damp_a(g, g->sx_i[i] + g->sz_i[k]) * p[o] - cp(g, k, i) * d;
        }
    }
    /* constitutive defect h delta(z - z_s) */
    if (hrow) {
        for (int j = 0; j < src->n; j++) {
            int i = src->i0 + j;
            double s = src->scale * hrow[j];
            p[(size_t)src->kp * NX + i] += cp(g, src->kp, i) * src->wp0 * s;
            if (src->wp1 != 0.0)
                p[(size_t)(src->kp + 1) * NX + i] += cp(g, src->kp + 1, i) * src->wp1 * s;
        }
    }
    /* traces: linear interpolation in z */
    if (prow) {
        for (int j = 0; j < rec->n; j++) {
            int i = rec->i0 + j;
            double s = rec->wp0 * p[(size_t)rec->kp * NX + i];
            if (rec->wp1 != 0.0) s += rec->wp1 * p[(size_t)(rec->kp + 1) * NX + i];
            prow[j] = s;
        }
    }
    if (vrow) {
        for (int j = 0; j < rec->n; j++) {
            int i = rec->i0 + j;
            double s = rec->wv0 * vz[(size_t)rec->kv * NX + i];
            if (rec->wv1 != 0.0) s += rec->wv1 * vz[(size_t)(rec->kv + 1) * NX + i];
            vrow[j] = s;
        }
    }
}

/* Transpose of og_step_fwd for step n (in place on the adjoint state).
 * On entry (pb, vxb, vzb) is the adjoint of (p^{n+1}, v^{n+1/2}) with the
 * adjoint of step n's sampling already added; on exit it is the adjoint of
 * (p^n, v^{n-1/2}). hbrow/fbrow receive the adjoint of step n's pressure /
 * velocity injection (or NULL). q and w are workspaces of NZ*NX doubles. */
void og_step_adj(const og_grid *g, double *pb, double *vxb, double *vzb,
                 const og_line *src, double *hbrow, double *fbrow,
                 double *q, double *wx, double *wz)
{
    const int NX = g->NX, NZ = g->NZ, R = g->R;
    /* transpose of the pressure half step */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int i = 0; i < NX; i++)
            q[(size_t)k * NX + i] = cp(g, k, i) * pb[(size_t)k * NX + i];
    if (hbrow) {
        for (int j = 0; j < src->n; j++) {
            int i = src->i0 + j;
            double s = src->wp0 * q[(size_t)src->kp * NX + i];
            if (src->wp1 != 0.0) s += src->wp1 * q[(size_t)(src->kp + 1) * NX + i];
            hbrow[j] = src->scale * s;
        }
    }
    /* vb += -(D-)^T q = D+ q ;  pb <- A_p pb */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++) {
        for (int j = 0; j < NX - 1; j++) {
            double d = 0.0;
            for (int m = 1; m <= R; m++)
                d += g->c[m - 1] * (P(g, q, k, j + m) - P(g, q, k, j - m + 1));
            vxb[(size_t)k * NX + j] += d;
        }
        if (k < NZ - 1) {
            for (int i = 0; i < NX; i++) {
                double d = 0.0;
                for (int m = 1; m <= R; m++)
                    d += g->c[m - 1] * (P(g, q, k + m, i) - P(g, q, k - m + 1, i));
                vzb[(size_t)k * NX + i] += d;
            }
        }
    }
    /* transpose of the velocity half step */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++) {
        for (int j = 0; j < NX - 1; j++)
            wx[(size_t)k * NX + j] = cvx(g, k, j) * vxb[(size_t)k * NX + j];
        wx[(size_t)k * NX + NX - 1] = 0.0;
        for (int i = 0; i < NX; i++)
            wz[(size_t)k * NX + i] = (k < NZ - 1) ? cvz(g, k, i) * vzb[(size_t)k * NX + i] : 0.0;
    }
    if (fbrow) {
        for (int j = 0; j < src->n; j++) {
            int i = src->i0 + j;
            double s = src->wv0 * wz[(size_t)src->kv * NX + i];
            if (src->wv1 != 0.0) s += src->wv1 * wz[(size_t)(src->kv + 1) * NX + i];
            fbrow[j] = src->scale * s;
        }
    }
    /* pb <- A_p pb - (D+)^T (C_v vb) = A_p pb + D- (C_v vb);  vb <- A_v vb */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++) {
        for (int i = 0; i < NX; i++) {
            double d = 0.0;
            for (int m = 1; m <= R; m++) {
                d += g->c[m - 1] * (VX(g, wx, k, i + m - 1) - VX(g, wx, k, i - m));
                d += g->c[m - 1] * (VZ(g, wz, k + m - 1, i) - VZ(g, wz, k - m, i));
            }
            size_t o = (size_t)k * NX + i;
            pb[o] = damp_a(g, g->sx_i[i] + g->sz_i[k]) * pb[o] + d;
        }
        for (int j = 0; j < NX - 1; j++) {
            size_t o = (size_t)k * NX + j;
            vxb[o] *= damp_a(g, g->sx_h[j] + g->sz_i[k]);
        }
        if (k < NZ - 1)
            for (int i = 0; i < NX; i++) {
                size_t o = (size_t)k * NX + i;
                vzb[o] *= damp_a(g, g->sx_i[i] + g->sz_h[k]);
            }
    }
}

/* Whole forward sweep from rest: the 2x2 modelling operator of eqn:fwd,
 * (h, f) on `src` -> (P p, P vz) on `rec`, gathers [nt][n] row-major. */
void og_forward(const og_grid *g, int nt, const og_line *src,
                const double *h, const double *f, const og_line *rec,
                double *outp, double *outv)
{
    size_t N = (size_t)g->NX * g->NZ;
    double *p = calloc(N, sizeof(double));
    double *vx = calloc(N, sizeof(double));
    double *vz = calloc(N, sizeof(double));
    for (int n = 0; n < nt; n++)
        og_step_fwd(g, p, vx, vz, src,
                    h ? h + (size_t)n * src->n : NULL,
                    f ? f + (size_t)n * src->n : NULL, rec,
                    outp ? outp + (size_t)n * rec->n : NULL,
                    outv ? outv + (size_t)n * rec->n : NULL);
    free(p); free(vx); free(vz);
}

/* Exact transpose of og_forward: (yp, yv) on `rec` -> (hb, fb) on `src`. */
void og_adjoint(const og_grid *g, int nt, const og_line *src,
                double *hb, double *fb, const og_line *rec,
                const double *yp, const double *yv)
{
    size_t N = (size_t)g->NX * g->NZ;
    const int NX = g->NX;
    double *pb = calloc(N, sizeof(double));
    double *vxb = calloc(N, sizeof(double));
    double *vzb = calloc(N, sizeof(double));
    double *q = calloc(N, sizeof(double));
    double *wx = calloc(N, sizeof(double));
    double *wz = calloc(N, sizeof(double));
    for (int n = nt - 1; n >= 0; n--) {
        /* transpose of step n's sampling: adjoint injection at the receivers */
        if (yp) {
            const double *row = yp + (size_t)n * rec->n;
            for (int j = 0; j < rec->n; j++) {
                int i = rec->i0 + j;
                pb[(size_t)rec->kp * NX + i] += rec->wp0 * row[j];
                if (rec->wp1 != 0.0) pb[(size_t)(rec->kp + 1) * NX + i] += rec->wp1 * row[j];
            }
        }
        if (yv) {
            const double *row = yv + (size_t)n * rec->n;
            for (int j = 0; j < rec->n; j++) {
                int i = rec->i0 + j;
                vzb[(size_t)rec->kv * NX + i] += rec->wv0 * row[j];
                if (rec->wv1 != 0.0) vzb[(size_t)(rec->kv + 1) * NX + i] += rec->wv1 * row[j];
            }
        }
        og_step_adj(g, pb, vxb, vzb, src,
                    hb ? hb + (size_t)n * src->n : NULL,
                    fb ? fb + (size_t)n * src->n : NULL, q, wx, wz);
    }
    free(pb); free(vxb); free(vzb); free(q); free(wx); free(wz);
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
