/*
 * FP64 CPU oracle of the sensor-misfit loss of a batch of walls and of its gradient with respect to
 * the material parameters, by the reverse-time (adjoint) sweep of the DF step. TEST INFRASTRUCTURE
 * ONLY (see hygro_oracle.h). The paper has no adjoint; what is differentiated is the DF step of
 * hygro_oracle.c exactly as written there ([eq:DF_NL], Pv first, then T with Pv^{n+1}; coefficients
 * of Sec. 2 at level n; arithmetic face means inside a layer, harmonic across layers; half-cell
 * Robin surfaces [eq:HAM_BC]), for walls without room faces.
 *
 * Loss: L = sum over samples k = 1..K (level m_k = k * sample_every), walls w and faces f of
 *   wT (T_f(m_k) - T_obs[k][w][f])^2 + wP (Pv_f(m_k) - P_obs[k][w][f])^2,
 * T_f, Pv_f the surface node values (node 0 for face 0, node N-1 for face 1).
 * Gradient: dL/dtheta for theta = the 9 affine-law parameters (kM0, a, cM0, b, kTT0, aT, cTT0, bT, chi)
 * of every layer.
 *
 * The reverse sweep stores every level of the forward run (no checkpointing: the oracle runs small
 * cases) and walks the steps backwards, applying the transposed Jacobian of each step to the adjoint
 * of the level it produced. A second, independent route gives directional derivatives: the forward
 * run in dual numbers (value, derivative along a direction of theta), orc_loss_tangent.
 */
#include "hygro_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { L_KM0, L_A, L_CM0, L_B, L_KTT0, L_AT, L_CTT0, L_BT, L_CHI };
enum { B_HT, B_HM, B_QINF, B_GINF };

typedef struct {
    double hT, hM, q, g, Tinf, Pinf;
} air_t;

/* the face data of wall w at time t (ambient or adiabatic faces) */
static air_t air_of(const orc_problem *p, int32_t w, int32_t f, double t)
{
    air_t a;
    memset(&a, 0, sizeof a);
    if (p->bc_kind[w * 2 + f] != ORC_BC_AMBIENT) return a;
    const double *b = p->bc_par + ((size_t)w * 2 + f) * ORC_NBC_PAR;
    a.hT = b[B_HT];
    a.hM = b[B_HM];
    a.q = b[B_QINF];
    a.g = b[B_GINF];
    orc_ambient(p, w, f, t, &a.Tinf, &a.Pinf);
    return a;
}

typedef struct {
    int32_t N, nl;
    double dx;
    const int32_t *first;
    const double *par;  /* [nl][9] */
    int32_t *layer;     /* [N] */
} wall_t;

static void wall_of(const orc_problem *p, const int64_t *loff, int32_t w, wall_t *v)
{
    v->N = p->n_nodes[w];
    v->nl = p->n_layers[w];
    v->dx = p->thickness[w] / (double)(v->N - 1);
    v->first = p->layer_first + loff[w];
    v->par = p->layer_par + (size_t)loff[w] * ORC_NLAYER_PAR;
    for (int32_t j = 0, l = 0; j < v->N; ++j) {
        while (l + 1 < v->nl && j >= v->first[l + 1]) ++l;
        v->layer[j] = l;
    }
}

/* ---- forward step (the formulas of hygro_oracle.c, wall_step) ------------------------------------ */

typedef struct {
    double *kM, *cM, *kTT, *cTT, *cTM, *kMf, *kTTf;   /* node [N] and face [N-1] values */
    double *Pn;
} fwd_t;

static void coefs(const orc_problem *p, const wall_t *v, const double *P, fwd_t *s)
{
    for (int32_t j = 0; j < v->N; ++j) {
        const double *q = v->par + (size_t)v->layer[j] * ORC_NLAYER_PAR;
        const double r = P[j] / p->Psat;
        s->kM[j] = q[L_KM0] * (1.0 + q[L_A] * r);
        s->cM[j] = q[L_CM0] * (1.0 + q[L_B] * r);
        s->kTT[j] = q[L_KTT0] * (1.0 + q[L_AT] * r);
        s->cTT[j] = q[L_CTT0] * (1.0 + q[L_BT] * r);
        s->cTM[j] = q[L_CHI] * s->cM[j];
    }
    for (int32_t j = 0; j + 1 < v->N; ++j) {
        if (v->layer[j] == v->layer[j + 1]) {
            s->kMf[j] = 0.5 * (s->kM[j] + s->kM[j + 1]);
            s->kTTf[j] = 0.5 * (s->kTT[j] + s->kTT[j + 1]);
        } else {
            s->kMf[j] = 2.0 * s->kM[j] * s->kM[j + 1] / (s->kM[j] + s->kM[j + 1]);
            s->kTTf[j] = 2.0 * s->kTT[j] * s->kTT[j + 1] / (s->kTT[j] + s->kTT[j + 1]);
        }
    }
}

/* levels n-1 (Tp, Pp) and n (Tc, Pc) -> n+1 (Tn, Pn) */
static void step(const orc_problem *p, const wall_t *v, const air_t a[2], const double *Tp, const double *Tc,
                 const double *Pp, const double *Pc, double *Tn, double *Pn, fwd_t *s)
{
    const int32_t N = v->N;
    const double dx = v->dx, dt = p->dt, Lv = p->Lv;
    coefs(p, v, Pc, s);
    for (int32_t j = 0; j < N; ++j) {
        const double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double A = w * dx * s->cM[j] / (2.0 * dt);
        double S = 0, nb = 0, H = 0, src = 0;
        if (j > 0) {
            S += s->kMf[j - 1] / dx;
            nb += s->kMf[j - 1] / dx * Pc[j - 1];
        }
        if (j < N - 1) {
            S += s->kMf[j] / dx;
            nb += s->kMf[j] / dx * Pc[j + 1];
        }
        if (j == 0) {
            H += a[0].hM;
            src += a[0].hM * a[0].Pinf + a[0].g;
        }
        if (j == N - 1) {
            H += a[1].hM;
            src += a[1].hM * a[1].Pinf + a[1].g;
        }
        Pn[j] = ((A - 0.5 * S - 0.5 * H) * Pp[j] + nb + src) / (A + 0.5 * S + 0.5 * H);
    }
    for (int32_t j = 0; j < N; ++j) {
        const double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double B = w * dx * s->cTT[j] / (2.0 * dt), C = w * dx * s->cTM[j] / (2.0 * dt);
        const double Pbar = 0.5 * (Pn[j] + Pp[j]);
        double S = 0, nb = 0, cross = 0, H = 0, src = 0;
        if (j > 0) {
            S += s->kTTf[j - 1] / dx;
            nb += s->kTTf[j - 1] / dx * Tc[j - 1];
            cross += Lv * s->kMf[j - 1] / dx * (Pc[j - 1] - Pbar);
        }
        if (j < N - 1) {
            S += s->kTTf[j] / dx;
            nb += s->kTTf[j] / dx * Tc[j + 1];
            cross += Lv * s->kMf[j] / dx * (Pc[j + 1] - Pbar);
        }
        for (int f = 0; f < 2; ++f)
            if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) {
                H += a[f].hT;
                src += a[f].hT * a[f].Tinf + Lv * a[f].hM * (a[f].Pinf - Pbar) + a[f].q;
            }
        Tn[j] = ((B - 0.5 * S - 0.5 * H) * Tp[j] + nb + cross + src - C * (Pn[j] - Pp[j])) / (B + 0.5 * S + 0.5 * H);
    }
}

/* ---- reverse of one step ----------------------------------------------------------------------------
 * Given lT, lP = dL/d(level n+1) (complete), add the contributions of this step to gTc, gPc (level n),
 * gTp, gPp (level n-1) and gpar (the wall's layers, [nl][9]). Every forward operation of step() is
 * reversed in the opposite order: T update, then Pv update, then the coefficients. */
typedef struct {
    double *gkM, *gcM, *gkTT, *gcTT, *gcTM, *gkMf, *gkTTf, *gPn;
} rev_t;

static void step_reverse(const orc_problem *p, const wall_t *v, const air_t a[2], const double *Tp,
                         const double *Tc, const double *Pp, const double *Pc, const double *Tn, const double *Pn,
                         const double *lT, const double *lP, double *gTp, double *gTc, double *gPp, double *gPc,
                         double *gpar, fwd_t *s, rev_t *r)
{
    const int32_t N = v->N;
    const double dx = v->dx, dt = p->dt, Lv = p->Lv, Ps = p->Psat;
    coefs(p, v, Pc, s);
    for (int32_t j = 0; j < N; ++j) {
        r->gkM[j] = r->gcM[j] = r->gkTT[j] = r->gcTT[j] = r->gcTM[j] = 0.0;
        r->gPn[j] = lP[j];
    }
    for (int32_t j = 0; j + 1 < N; ++j) r->gkMf[j] = r->gkTTf[j] = 0.0;

    /* T update: Tn = NumT / DenT */
    for (int32_t j = 0; j < N; ++j) {
        const double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double B = w * dx * s->cTT[j] / (2.0 * dt), C = w * dx * s->cTM[j] / (2.0 * dt);
        const double Pbar = 0.5 * (Pn[j] + Pp[j]);
        double S = 0, H = 0;
        if (j > 0) S += s->kTTf[j - 1] / dx;
        if (j < N - 1) S += s->kTTf[j] / dx;
        if (j == 0) H += a[0].hT;
        if (j == N - 1) H += a[1].hT;
        const double Den = B + 0.5 * S + 0.5 * H;
        const double gNum = lT[j] / Den, gDen = -lT[j] * Tn[j] / Den;
        double gB = gNum * Tp[j] + gDen;
        double gS = -0.5 * gNum * Tp[j] + 0.5 * gDen;
        double gPbar = 0.0;
        gTp[j] += gNum * (B - 0.5 * S - 0.5 * H);
        if (j > 0) {
            r->gkTTf[j - 1] += (gNum * Tc[j - 1] + gS) / dx;
            gTc[j - 1] += gNum * s->kTTf[j - 1] / dx;
            r->gkMf[j - 1] += gNum * Lv * (Pc[j - 1] - Pbar) / dx;
            gPc[j - 1] += gNum * Lv * s->kMf[j - 1] / dx;
            gPbar -= gNum * Lv * s->kMf[j - 1] / dx;
        }
        if (j < N - 1) {
            r->gkTTf[j] += (gNum * Tc[j + 1] + gS) / dx;
            gTc[j + 1] += gNum * s->kTTf[j] / dx;
            r->gkMf[j] += gNum * Lv * (Pc[j + 1] - Pbar) / dx;
            gPc[j + 1] += gNum * Lv * s->kMf[j] / dx;
            gPbar -= gNum * Lv * s->kMf[j] / dx;
        }
        for (int f = 0; f < 2; ++f)
            if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) gPbar -= gNum * Lv * a[f].hM;
        const double gC = -gNum * (Pn[j] - Pp[j]);
        r->gPn[j] += -gNum * C + 0.5 * gPbar;
        gPp[j] += gNum * C + 0.5 * gPbar;
        r->gcTT[j] += gB * w * dx / (2.0 * dt);
        r->gcTM[j] += gC * w * dx / (2.0 * dt);
    }
    /* Pv update: Pn = Num / Den */
    for (int32_t j = 0; j < N; ++j) {
        const double w = (j == 0 || j == N - 1) ? 0.5 : 1.0;
        const double A = w * dx * s->cM[j] / (2.0 * dt);
        double S = 0, H = 0;
        if (j > 0) S += s->kMf[j - 1] / dx;
        if (j < N - 1) S += s->kMf[j] / dx;
        if (j == 0) H += a[0].hM;
        if (j == N - 1) H += a[1].hM;
        const double Den = A + 0.5 * S + 0.5 * H;
        const double gNum = r->gPn[j] / Den, gDen = -r->gPn[j] * Pn[j] / Den;
        const double gA = gNum * Pp[j] + gDen;
        const double gS = -0.5 * gNum * Pp[j] + 0.5 * gDen;
        gPp[j] += gNum * (A - 0.5 * S - 0.5 * H);
        if (j > 0) {
            r->gkMf[j - 1] += (gNum * Pc[j - 1] + gS) / dx;
            gPc[j - 1] += gNum * s->kMf[j - 1] / dx;
        }
        if (j < N - 1) {
            r->gkMf[j] += (gNum * Pc[j + 1] + gS) / dx;
            gPc[j + 1] += gNum * s->kMf[j] / dx;
        }
        r->gcM[j] += gA * w * dx / (2.0 * dt);
    }
    /* face values */
    for (int32_t j = 0; j + 1 < N; ++j) {
        if (v->layer[j] == v->layer[j + 1]) {
            r->gkM[j] += 0.5 * r->gkMf[j];
            r->gkM[j + 1] += 0.5 * r->gkMf[j];
            r->gkTT[j] += 0.5 * r->gkTTf[j];
            r->gkTT[j + 1] += 0.5 * r->gkTTf[j];
        } else {
            double x = s->kM[j], y = s->kM[j + 1], d = (x + y) * (x + y);
            r->gkM[j] += r->gkMf[j] * 2.0 * y * y / d;
            r->gkM[j + 1] += r->gkMf[j] * 2.0 * x * x / d;
            x = s->kTT[j];
            y = s->kTT[j + 1];
            d = (x + y) * (x + y);
            r->gkTT[j] += r->gkTTf[j] * 2.0 * y * y / d;
            r->gkTT[j + 1] += r->gkTTf[j] * 2.0 * x * x / d;
        }
    }
    /* node coefficients of Sec. 2 (cTM = chi cM first, it feeds cM's adjoint) */
    for (int32_t j = 0; j < N; ++j) {
        const double *q = v->par + (size_t)v->layer[j] * ORC_NLAYER_PAR;
        double *g = gpar + (size_t)v->layer[j] * ORC_NLAYER_PAR;
        const double rr = Pc[j] / Ps;
        g[L_CHI] += r->gcTM[j] * s->cM[j];
        r->gcM[j] += r->gcTM[j] * q[L_CHI];
        g[L_KM0] += r->gkM[j] * (1.0 + q[L_A] * rr);
        g[L_A] += r->gkM[j] * q[L_KM0] * rr;
        g[L_CM0] += r->gcM[j] * (1.0 + q[L_B] * rr);
        g[L_B] += r->gcM[j] * q[L_CM0] * rr;
        g[L_KTT0] += r->gkTT[j] * (1.0 + q[L_AT] * rr);
        g[L_AT] += r->gkTT[j] * q[L_KTT0] * rr;
        g[L_CTT0] += r->gcTT[j] * (1.0 + q[L_BT] * rr);
        g[L_BT] += r->gcTT[j] * q[L_CTT0] * rr;
        gPc[j] += (r->gkM[j] * q[L_KM0] * q[L_A] + r->gcM[j] * q[L_CM0] * q[L_B] + r->gkTT[j] * q[L_KTT0] * q[L_AT] +
                   r->gcTT[j] * q[L_CTT0] * q[L_BT]) /
                  Ps;
    }
}

static int64_t *layer_offsets(const orc_problem *p)
{
    int64_t *off = (int64_t *)calloc((size_t)p->n_walls + 1, sizeof(int64_t));
    if (off)
        for (int32_t i = 0; i < p->n_walls; ++i) off[i + 1] = off[i] + p->n_layers[i];
    return off;
}

/* misfit of one wall at one sample level: adds to *loss, and (if gT / gP) its derivative at the surface nodes */
static void misfit(const orc_misfit *m, int32_t W, int32_t w, int32_t k, int32_t N, const double *T, const double *P,
                   double *loss, double *gT, double *gP)
{
    for (int f = 0; f < 2; ++f) {
        const int32_t j = f == 0 ? 0 : N - 1;
        const double *o = m->obs + (((size_t)k * W + w) * 2 + f) * 2;
        const double eT = T[j] - o[0], eP = P[j] - o[1];
        *loss += m->wT * eT * eT + m->wP * eP * eP;
        if (gT) gT[j] += 2.0 * m->wT * eT;
        if (gP) gP[j] += 2.0 * m->wP * eP;
    }
}

int orc_loss_adjoint(const orc_problem *p, int64_t n_steps, const orc_misfit *m, double *loss_out, double *grad,
                     int32_t n_threads)
{
    if (p == NULL || m == NULL || loss_out == NULL || n_steps < 0 || m->sample_every < 1) return -1;
    if (p->n_rooms > 0) return -1;
    if (p->layer_law != NULL) {   /* the adjoint differentiates the affine laws only */
        int64_t nl = 0;
        for (int32_t w = 0; w < p->n_walls; ++w) nl += p->n_layers[w];
        for (int64_t l = 0; l < nl; ++l)
            if (p->layer_law[l] != ORC_LAW_AFFINE) return -1;
    }
    if (p->vapour_frac != NULL)
        for (int32_t w = 0; w < p->n_walls; ++w)
            if (p->vapour_frac[w] != 1.0) return -1;   /* the adjoint takes kTM = Lv kM */
    int64_t *loff = layer_offsets(p);
    if (loff == NULL) return -2;
    const int64_t total_layers = loff[p->n_walls];
    if (grad) memset(grad, 0, sizeof(double) * (size_t)total_layers * ORC_NLAYER_PAR);
    const int32_t K = (int32_t)(n_steps / m->sample_every);
    if (n_threads <= 0) n_threads = 1;
    double loss = 0.0;
    int rc = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1) reduction(+ : loss)
#endif
    for (int32_t w = 0; w < p->n_walls; ++w) {
        const int32_t N = p->n_nodes[w];
        const size_t lev = (size_t)(n_steps + 1) * N;
        double *T = (double *)malloc(sizeof(double) * lev), *P = (double *)malloc(sizeof(double) * lev);
        double *buf = (double *)malloc(sizeof(double) * (size_t)N * 24);
        int32_t *layer = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
        if (!T || !P || !buf || !layer) {
            free(T);
            free(P);
            free(buf);
            free(layer);
#ifdef _OPENMP
#pragma omp atomic write
#endif
            rc = -2;
            continue;
        }
        wall_t v;
        v.layer = layer;
        wall_of(p, loff, w, &v);
        fwd_t s = {buf, buf + N, buf + 2 * N, buf + 3 * N, buf + 4 * N, buf + 5 * N, buf + 6 * N, buf + 7 * N};
        rev_t r = {buf + 8 * N, buf + 9 * N, buf + 10 * N, buf + 11 * N, buf + 12 * N, buf + 13 * N, buf + 14 * N,
                   buf + 15 * N};
        double *lT = buf + 16 * N, *lP = buf + 17 * N, *mT = buf + 18 * N, *mP = buf + 19 * N;
        double *nT = buf + 20 * N, *nP = buf + 21 * N;
        /* level 0: the wall's uniform initial state ([eq:HAM_ic]) */
        for (int32_t j = 0; j < N; ++j) {
            T[j] = m->T_init[w];
            P[j] = m->P_init[w];
        }
        double lw = 0.0;
        /* forward, every level stored; level -1 := level 0 */
        for (int64_t n = 0; n < n_steps; ++n) {
            const double t = p->t0 + (double)n * p->dt;
            const air_t a[2] = {air_of(p, w, 0, t), air_of(p, w, 1, t)};
            const double *Tc = T + (size_t)n * N, *Pc = P + (size_t)n * N;
            const double *Tp = n > 0 ? Tc - N : Tc, *Pp = n > 0 ? Pc - N : Pc;
            step(p, &v, a, Tp, Tc, Pp, Pc, T + (size_t)(n + 1) * N, P + (size_t)(n + 1) * N, &s);
            if ((n + 1) % m->sample_every == 0 && (n + 1) / m->sample_every <= K)
                misfit(m, p->n_walls, w, (int32_t)((n + 1) / m->sample_every - 1), N, T + (size_t)(n + 1) * N,
                       P + (size_t)(n + 1) * N, &lw, NULL, NULL);
        }
        loss += lw;
        if (grad) {
            double *g = grad + (size_t)loff[w] * ORC_NLAYER_PAR;
            /* l = adjoint of level n+1 (complete), mm = partial adjoint of level n */
            for (int32_t j = 0; j < N; ++j) lT[j] = lP[j] = mT[j] = mP[j] = 0.0;
            if (n_steps > 0 && n_steps % m->sample_every == 0 && n_steps / m->sample_every <= K) {
                double dummy = 0.0;
                misfit(m, p->n_walls, w, (int32_t)(n_steps / m->sample_every - 1), N, T + (size_t)n_steps * N,
                       P + (size_t)n_steps * N, &dummy, lT, lP);
            }
            for (int64_t n = n_steps - 1; n >= 0; --n) {
                const double t = p->t0 + (double)n * p->dt;
                const air_t a[2] = {air_of(p, w, 0, t), air_of(p, w, 1, t)};
                const double *Tc = T + (size_t)n * N, *Pc = P + (size_t)n * N;
                const double *Tp = n > 0 ? Tc - N : Tc, *Pp = n > 0 ? Pc - N : Pc;
                /* the partial adjoint of level n-1 starts empty; level n's own sample term joins its
                   partial adjoint before this step's contributions complete it */
                for (int32_t j = 0; j < N; ++j) nT[j] = nP[j] = 0.0;
                if (n >= 1 && n % m->sample_every == 0 && n / m->sample_every <= K) {
                    double dummy = 0.0;
                    misfit(m, p->n_walls, w, (int32_t)(n / m->sample_every - 1), N, Tc, Pc, &dummy, mT, mP);
                }
                if (n > 0) {
                    step_reverse(p, &v, a, Tp, Tc, Pp, Pc, Tc + N, Pc + N, lT, lP, nT, mT, nP, mP, g, &s, &r);
                } else {
                    /* the first step reads level 0 as both n and n-1 */
                    step_reverse(p, &v, a, Tc, Tc, Pc, Pc, Tc + N, Pc + N, lT, lP, mT, mT, mP, mP, g, &s, &r);
                }
                /* shift: level n is complete now; level n-1 keeps its partial */
                for (int32_t j = 0; j < N; ++j) {
                    lT[j] = mT[j];
                    lP[j] = mP[j];
                    mT[j] = nT[j];
                    mP[j] = nP[j];
                }
            }
        }
        free(T);
        free(P);
        free(buf);
        free(layer);
    }
    free(loff);
    *loss_out = loss;
    return rc;
}

/* ---- forward mode: the same run in dual numbers ------------------------------------------------------ */

typedef struct {
    double v, d;
} dual;

static inline dual D(double v) { return (dual){v, 0.0}; }
static inline dual dadd(dual a, dual b) { return (dual){a.v + b.v, a.d + b.d}; }
static inline dual dsub(dual a, dual b) { return (dual){a.v - b.v, a.d - b.d}; }
static inline dual dmul(dual a, dual b) { return (dual){a.v * b.v, a.d * b.v + a.v * b.d}; }
static inline dual ddiv(dual a, dual b) { return (dual){a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
static inline dual dscale(double s, dual a) { return (dual){s * a.v, s * a.d}; }

int orc_loss_tangent(const orc_problem *p, int64_t n_steps, const orc_misfit *m, const double *dir, double *loss_out,
                     double *dloss_out)
{
    if (p == NULL || m == NULL || dir == NULL || n_steps < 0 || m->sample_every < 1 || p->n_rooms > 0) return -1;
    if (p->layer_law != NULL) {   /* affine laws only, as the reverse sweep */
        int64_t nl = 0;
        for (int32_t w = 0; w < p->n_walls; ++w) nl += p->n_layers[w];
        for (int64_t l = 0; l < nl; ++l)
            if (p->layer_law[l] != ORC_LAW_AFFINE) return -1;
    }
    if (p->vapour_frac != NULL)
        for (int32_t w = 0; w < p->n_walls; ++w)
            if (p->vapour_frac[w] != 1.0) return -1;
    int64_t *loff = layer_offsets(p);
    if (loff == NULL) return -2;
    const int32_t K = (int32_t)(n_steps / m->sample_every);
    const double dt = p->dt, Lv = p->Lv, Ps = p->Psat;
    dual L = D(0.0);
    for (int32_t w = 0; w < p->n_walls; ++w) {
        const int32_t N = p->n_nodes[w];
        const int32_t nl = p->n_layers[w];
        const double dx = p->thickness[w] / (double)(N - 1);
        dual *buf = (dual *)malloc(sizeof(dual) * (size_t)N * 11);
        dual *par = (dual *)malloc(sizeof(dual) * (size_t)nl * ORC_NLAYER_PAR);
        int32_t *layer = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
        if (!buf || !par || !layer) {
            free(buf);
            free(par);
            free(layer);
            free(loff);
            return -2;
        }
        for (int32_t i = 0; i < nl * ORC_NLAYER_PAR; ++i) {
            par[i].v = p->layer_par[(size_t)loff[w] * ORC_NLAYER_PAR + i];
            par[i].d = dir[(size_t)loff[w] * ORC_NLAYER_PAR + i];
        }
        for (int32_t j = 0, l = 0; j < N; ++j) {
            while (l + 1 < nl && j >= p->layer_first[loff[w] + l + 1]) ++l;
            layer[j] = l;
        }
        dual *Tp = buf, *Tc = buf + N, *Pp = buf + 2 * N, *Pc = buf + 3 * N, *Tn = buf + 4 * N, *Pn = buf + 5 * N;
        dual *kM = buf + 6 * N, *cM = buf + 7 * N, *kTT = buf + 8 * N, *cTT = buf + 9 * N, *cTM = buf + 10 * N;
        for (int32_t j = 0; j < N; ++j) {
            Tp[j] = Tc[j] = D(m->T_init[w]);
            Pp[j] = Pc[j] = D(m->P_init[w]);
        }
        for (int64_t n = 0; n < n_steps; ++n) {
            const double t = p->t0 + (double)n * dt;
            const air_t a[2] = {air_of(p, w, 0, t), air_of(p, w, 1, t)};
            for (int32_t j = 0; j < N; ++j) {
                const dual *q = par + (size_t)layer[j] * ORC_NLAYER_PAR;
                const dual rr = dscale(1.0 / Ps, Pc[j]);
                kM[j] = dmul(q[L_KM0], dadd(D(1.0), dmul(q[L_A], rr)));
                cM[j] = dmul(q[L_CM0], dadd(D(1.0), dmul(q[L_B], rr)));
                kTT[j] = dmul(q[L_KTT0], dadd(D(1.0), dmul(q[L_AT], rr)));
                cTT[j] = dmul(q[L_CTT0], dadd(D(1.0), dmul(q[L_BT], rr)));
                cTM[j] = dmul(q[L_CHI], cM[j]);
            }
            /* face value between j and j+1 */
#define FACE(k, j) (layer[j] == layer[(j) + 1] ? dscale(0.5, dadd(k[j], k[(j) + 1]))                              \
                                                 : ddiv(dscale(2.0, dmul(k[j], k[(j) + 1])), dadd(k[j], k[(j) + 1])))
            for (int32_t j = 0; j < N; ++j) {
                const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
                const dual A = dscale(wj * dx / (2.0 * dt), cM[j]);
                dual S = D(0), nb = D(0), H = D(0), src = D(0);
                if (j > 0) {
                    const dual F = dscale(1.0 / dx, FACE(kM, j - 1));
                    S = dadd(S, F);
                    nb = dadd(nb, dmul(F, Pc[j - 1]));
                }
                if (j < N - 1) {
                    const dual F = dscale(1.0 / dx, FACE(kM, j));
                    S = dadd(S, F);
                    nb = dadd(nb, dmul(F, Pc[j + 1]));
                }
                if (j == 0) {
                    H = dadd(H, D(a[0].hM));
                    src = dadd(src, D(a[0].hM * a[0].Pinf + a[0].g));
                }
                if (j == N - 1) {
                    H = dadd(H, D(a[1].hM));
                    src = dadd(src, D(a[1].hM * a[1].Pinf + a[1].g));
                }
                const dual hs = dscale(0.5, dadd(S, H));
                Pn[j] = ddiv(dadd(dadd(dmul(dsub(A, hs), Pp[j]), nb), src), dadd(A, hs));
            }
            for (int32_t j = 0; j < N; ++j) {
                const double wj = (j == 0 || j == N - 1) ? 0.5 : 1.0;
                const dual B = dscale(wj * dx / (2.0 * dt), cTT[j]), C = dscale(wj * dx / (2.0 * dt), cTM[j]);
                const dual Pbar = dscale(0.5, dadd(Pn[j], Pp[j]));
                dual S = D(0), nb = D(0), cross = D(0), H = D(0), src = D(0);
                if (j > 0) {
                    const dual F = dscale(1.0 / dx, FACE(kTT, j - 1));
                    S = dadd(S, F);
                    nb = dadd(nb, dmul(F, Tc[j - 1]));
                    cross = dadd(cross, dmul(dscale(Lv / dx, FACE(kM, j - 1)), dsub(Pc[j - 1], Pbar)));
                }
                if (j < N - 1) {
                    const dual F = dscale(1.0 / dx, FACE(kTT, j));
                    S = dadd(S, F);
                    nb = dadd(nb, dmul(F, Tc[j + 1]));
                    cross = dadd(cross, dmul(dscale(Lv / dx, FACE(kM, j)), dsub(Pc[j + 1], Pbar)));
                }
                for (int f = 0; f < 2; ++f)
                    if ((f == 0 && j == 0) || (f == 1 && j == N - 1)) {
                        H = dadd(H, D(a[f].hT));
                        src = dadd(src, dadd(D(a[f].hT * a[f].Tinf + a[f].q),
                                             dscale(Lv * a[f].hM, dsub(D(a[f].Pinf), Pbar))));
                    }
                const dual hs = dscale(0.5, dadd(S, H));
                const dual num = dsub(dadd(dadd(dadd(dmul(dsub(B, hs), Tp[j]), nb), cross), src),
                                      dmul(C, dsub(Pn[j], Pp[j])));
                Tn[j] = ddiv(num, dadd(B, hs));
            }
#undef FACE
            for (int32_t j = 0; j < N; ++j) {
                Tp[j] = Tc[j];
                Pp[j] = Pc[j];
                Tc[j] = Tn[j];
                Pc[j] = Pn[j];
            }
            if ((n + 1) % m->sample_every == 0 && (n + 1) / m->sample_every <= K) {
                const int32_t k = (int32_t)((n + 1) / m->sample_every - 1);
                for (int f = 0; f < 2; ++f) {
                    const int32_t j = f == 0 ? 0 : N - 1;
                    const double *o = m->obs + (((size_t)k * p->n_walls + w) * 2 + f) * 2;
                    const dual eT = dsub(Tc[j], D(o[0])), eP = dsub(Pc[j], D(o[1]));
                    L = dadd(L, dadd(dscale(m->wT, dmul(eT, eT)), dscale(m->wP, dmul(eP, eP))));
                }
            }
        }
        free(buf);
        free(par);
        free(layer);
    }
    free(loff);
    *loss_out = L.v;
    *dloss_out = L.d;
    return 0;
}
