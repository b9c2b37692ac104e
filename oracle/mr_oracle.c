/*
 * mr_oracle.c -- plain FP64 CPU oracle of MR + MRLT/NERK (arXiv 1905.08717).
 *
 * TEST INFRASTRUCTURE ONLY (see mr_oracle.h).  Deliberately simple and slow:
 * every level l keeps dense arrays over all 2^{d l} cells, a node status per
 * cell (0 absent, 1 leaf, 2 internal node), and every loop visits cells in
 * index order.  Each routine names the passage of the paper it follows.
 * Values are stored the way the paper stores them (compact RK stages plus the
 * NERK partial sums, Sec. 3 "Compact formulation").  Readings of passages the
 * paper leaves open are marked READING and are listed in the design notes.
 *
 * Parity unpinned (no test outside this file can fix it):
 *  - beta = 1/8 in the AUSM+ Mach splitting (ausm_mach): taken as Liou (1996)
 *    publishes it; the other AUSM+ terms are pinned by the flux tests.
 * The internal-child values of the stage-2/3 projections (Eq. 15, Alg. 6) reach
 * no leaf value on a graded tree with radius-2 stencils; they are read back
 * through OR_READ_NODES and pinned on a profile whose exact solution is linear
 * in time (every stored value then equals the exact one at its instant).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * same source gives the same bits on x86-64 and aarch64).
 */
#include "mr_oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define LMAX 16
#define MMAX 5

typedef struct {
    or_config cfg;
    int d, m, L, lb, eq, rk, gts, nf;
    int n[LMAX + 1];
    long nc[LMAX + 1];
    double dx[LMAX + 1][3];
    double vol[LMAX + 1];
    unsigned char* st[LMAX + 1];
    /* per-node storage, AoS [cell][var] */
    double *Q0[LMAX + 1], *Q1[LMAX + 1], *Q2[LMAX + 1], *QE[LMAX + 1];
    double *XH[LMAX + 1], *NH[LMAX + 1], *N1[LMAX + 1], *N3[LMAX + 1], *QX[LMAX + 1];
    double *RC[LMAX + 1], *RF[LMAX + 1]; /* [cell][2d faces][var] */
    double scale[MMAX];
    double t, dt;
    long long iters, macros, updates, near;
    long long pos; /* next iteration index within the current macro step */
    int bad;
    char err[256];
} Orc;

/* exposure context: level u being updated, stage s (0 = plain q^n of every
 * node, used by the adaptation), coarsest active level lmin */
typedef struct {
    int u, s, lmin;
} Ctx;

static void fail(Orc* o, const char* fmt, ...)
{
    if (o->bad) return;
    o->bad = 1;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(o->err, sizeof o->err, fmt, ap);
    va_end(ap);
}

/* ------------------------------------------------------------ indexing */
static long lin(const Orc* o, int l, const int c[3])
{
    long n = o->n[l];
    return c[0] + n * ((long)c[1] + n * (long)c[2]);
}

static void coords(const Orc* o, int l, long id, int c[3])
{
    long n = o->n[l];
    c[0] = (int)(id % n);
    c[1] = (int)((id / n) % n);
    c[2] = (int)(id / (n * n));
    if (o->d < 3) c[2] = 0;
    if (o->d < 2) c[1] = 0;
}

/* ghost rule (the paper states boundary conditions only for the PDE; the
 * same rule is used on every level): periodic wrap; homogeneous Neumann as an
 * even mirror about the wall; zero Dirichlet as an odd mirror, the ghost
 * taking the negated value, so that *sgn changes sign at every reflection on
 * a Dirichlet wall. */
static int mirror_s(const Orc* o, int l, int k, int p, double* sgn)
{
    int n = o->n[l];
    if (o->cfg.bc[k] == 0) {
        p %= n;
        if (p < 0) p += n;
        return p;
    }
    while (p < 0 || p >= n) {
        if (p < 0) p = -1 - p;
        else p = 2 * n - 1 - p;
        if (o->cfg.bc[k] == 2) *sgn = -*sgn;
    }
    return p;
}

/* neighbourhood map for tree rules: periodic wrap, walls drop the cell */
static int inside(const Orc* o, int l, int k, int p, int* q)
{
    int n = o->n[l];
    if (o->cfg.bc[k] == 0) {
        p %= n;
        if (p < 0) p += n;
        *q = p;
        return 1;
    }
    if (p < 0 || p >= n) return 0;
    *q = p;
    return 1;
}

#define V(F, l, id) ((F)[l] + (long)(id) * o->m)

/* ------------------------------------------------------------ exposures */
/* Value a stored node (leaf or internal) of level l shows to the stencil of
 * a level-u leaf at stage s of the current LT iteration.  This is the table
 * of Secs. 4.1-4.3 and Algs. 3-9:
 *   same level (l = u):  q^n, q*, q** at stages 1, 2, 3; internal nodes carry
 *     the projections of Alg. 3 (stage 1), Alg. 4 (stage 2), Alg. 6 (stage 3).
 *   finer level (l = u+1, coarse-fine faces computed with virtual children,
 *     Sec. 2 flux scenarios): stage 1 q^n; stage 2 the extrapolations to
 *     t^n + 2 dt_{l}: leaves Eq. 14, internal nodes Eq. 15; stage 3 the value
 *     at t^n + dt_l: leaves q^{n+1}, internal nodes Eq. 16 (Alg. 6).
 *   coarser level l = u-1 >= lmin (source of virtual cells, Alg. 8/9):
 *     stage 1 q^n; stage 2 the half-step value (leaves q^n + k1/2, Sec. 4.1.1;
 *     internal nodes Eq. 17); stage 3 the NERK theta=1/4 value (Alg. 9).
 *   coarser level l = lmin-1 (mid-step, Alg. 3 and Sec. 4.3): stage 1 the
 *     theta=1/2 value (RK2 NERK, RK3 q**); stage 2 the end value q^{n+1}
 *     (internal nodes Eq. 22 / Eq. 16); stage 3 the NERK theta=3/4 value. */
static void expose(Orc* o, int l, long id, const Ctx* x, double* out)
{
    int m = o->m, v;
    unsigned char s = o->st[l][id];
    const double *a = NULL, *b = NULL;
    int rel = l - x->u;
    if (s == 0) {
        fail(o, "expose: absent node level %d cell %ld", l, id);
        for (v = 0; v < m; v++) out[v] = 0.0;
        return;
    }
    if (x->s == 0 || (x->s == 1 && o->gts)) {
        a = V(o->Q0, l, id);
    } else if (o->gts) {
        a = x->s == 2 ? V(o->Q1, l, id) : V(o->Q2, l, id);
    } else if (rel < -1 || rel > 1 || (rel == -1 && l < x->lmin - 1)) {
        fail(o, "expose: level %d seen from level %d (lmin %d)", l, x->u, x->lmin);
        for (v = 0; v < m; v++) out[v] = 0.0;
        return;
    } else if (x->s == 1) {
        if (rel >= 0 || l >= x->lmin) a = V(o->Q0, l, id);
        else a = o->rk == 2 ? V(o->NH, l, id) : V(o->Q2, l, id);
    } else if (x->s == 2) {
        if (rel == 0) a = V(o->Q1, l, id);
        else if (rel == 1) {
            if (s == 1) a = V(o->QX, l, id);
            else { /* Eq. 15: 2 q* - q^n of an internal node */
                a = V(o->Q1, l, id);
                b = V(o->Q0, l, id);
                for (v = 0; v < m; v++) out[v] = 2.0 * a[v] - b[v];
                return;
            }
        } else if (l >= x->lmin) {
            if (s == 1) { /* Sec. 4.1.1: first-order q^n + a21 k1 / 2 */
                a = V(o->Q0, l, id);
                b = V(o->Q1, l, id);
                for (v = 0; v < m; v++) out[v] = a[v] + 0.5 * (b[v] - a[v]);
                return;
            }
            a = V(o->XH, l, id);
        } else a = V(o->QE, l, id);
    } else {
        if (rel == 0) a = V(o->Q2, l, id);
        else if (rel == 1) a = V(o->QE, l, id);
        else if (l >= x->lmin) a = V(o->N1, l, id);
        else a = V(o->N3, l, id);
    }
    for (v = 0; v < m; v++) out[v] = a[v];
}

/* Prediction of a cell of level l from its parent level (Eq. 4a/4b), applied
 * as a tensor product in 2D/3D (READING: the paper defers the 2D/3D operators
 * to its reference RSTB03): the 1D rule is applied along x, then y, then z on
 * the 3^d block of parent-level values around the parent. */
static void predict_cell(Orc* o, int l, const int q[3], const Ctx* x, double* out)
{
    int d = o->d, m = o->m, v, k;
    double B[27][MMAX];
    int P[3] = {0, 0, 0}, a[3] = {0, 0, 0};
    if (l - 1 < o->lb) {
        fail(o, "predict: level %d has no parent level", l);
        for (v = 0; v < m; v++) out[v] = 0.0;
        return;
    }
    for (k = 0; k < d; k++) {
        P[k] = q[k] >> 1;
        a[k] = q[k] & 1;
    }
    int dz, dy, dxx;
    for (dz = -1; dz <= 1; dz++)
        for (dy = -1; dy <= 1; dy++)
            for (dxx = -1; dxx <= 1; dxx++) {
                int idx = (dz + 1) * 9 + (dy + 1) * 3 + (dxx + 1);
                if ((d < 3 && dz != 0) || (d < 2 && dy != 0)) continue;
                int p[3] = {0, 0, 0}, off[3] = {dxx, dy, dz};
                double sg = 1.0;
                for (k = 0; k < d; k++) p[k] = mirror_s(o, l - 1, k, P[k] + off[k], &sg);
                long id = lin(o, l - 1, p);
                if (o->st[l - 1][id] == 0) {
                    fail(o, "predict: source (%d,%d,%d) at level %d absent", p[0], p[1], p[2], l - 1);
                    for (v = 0; v < m; v++) B[idx][v] = 0.0;
                    continue;
                }
                expose(o, l - 1, id, x, B[idx]);
                if (sg < 0.0)
                    for (v = 0; v < m; v++) B[idx][v] = -B[idx][v];
            }
    /* collapse along x */
    double R[9][MMAX];
    for (dz = -1; dz <= 1; dz++)
        for (dy = -1; dy <= 1; dy++) {
            if ((d < 3 && dz != 0) || (d < 2 && dy != 0)) continue;
            int base = (dz + 1) * 9 + (dy + 1) * 3;
            int r = (dz + 1) * 3 + (dy + 1);
            for (v = 0; v < m; v++) {
                double c = B[base + 1][v], dm = B[base + 2][v] - B[base][v];
                R[r][v] = a[0] ? c + dm / 8.0 : c - dm / 8.0;
            }
        }
    if (d == 1) {
        for (v = 0; v < m; v++) out[v] = R[4][v];
        return;
    }
    /* collapse along y */
    double S[3][MMAX];
    for (dz = -1; dz <= 1; dz++) {
        if (d < 3 && dz != 0) continue;
        for (v = 0; v < m; v++) {
            double c = R[(dz + 1) * 3 + 1][v];
            double dm = R[(dz + 1) * 3 + 2][v] - R[(dz + 1) * 3][v];
            S[dz + 1][v] = a[1] ? c + dm / 8.0 : c - dm / 8.0;
        }
    }
    if (d == 2) {
        for (v = 0; v < m; v++) out[v] = S[1][v];
        return;
    }
    for (v = 0; v < m; v++) {
        double c = S[1][v], dm = S[2][v] - S[0][v];
        out[v] = a[2] ? c + dm / 8.0 : c - dm / 8.0;
    }
}

/* value of the cell at (possibly out-of-box) coordinates p of level l: ghost
 * rule, then the stored node's exposure or, for a virtual cell, a prediction
 * from the parent level (Sec. 2, virtual leaves). */
static void value_at(Orc* o, int l, const int p[3], const Ctx* x, double* out)
{
    int q[3] = {0, 0, 0}, k, v;
    double sg = 1.0;
    for (k = 0; k < o->d; k++) q[k] = mirror_s(o, l, k, p[k], &sg);
    long id = lin(o, l, q);
    if (o->st[l][id]) expose(o, l, id, x, out);
    else predict_cell(o, l, q, x, out);
    if (sg < 0.0)
        for (v = 0; v < o->m; v++) out[v] = -out[v];
}

/* ------------------------------------------------------------ physics */
static double minmod(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/* AUSM+ flux (Liou, J. Comput. Phys. 129, 1996), the paper's flux for the
 * Euler equations (Sec. 5), from the reconstructed primitive states PL, PR
 * (rho, velocities, p) and conservative states UL, UR, across a face normal
 * to direction k:
 *   critical speed a*^2 = 2 (g-1)/(g+1) H, H = (E + p)/rho;
 *   interface speed a = min(a*_L^2 / max(a*_L, u_L), a*_R^2 / max(a*_R, -u_R));
 *   M_L = u_L / a, M_R = u_R / a (normal velocities);
 *   Mach splitting M+-(M) = +-(M +- 1)^2/4 +- beta (M^2 - 1)^2 for |M| < 1,
 *     else (M +- |M|)/2, beta = 1/8;
 *   pressure splitting P+-(M) = (M +- 1)^2 (2 -+ M)/4 +- alpha M (M^2 - 1)^2
 *     for |M| < 1, else (1 +- sign M)/2, alpha = 3/16;
 *   m = M+(M_L) + M-(M_R), p_half = P+(M_L) p_L + P-(M_R) p_R;
 *   F = a (max(m,0) Psi_L + min(m,0) Psi_R) + p_half n, Psi = rho (1, u, H). */
static double ausm_mach(double M, int sgn)
{
    if (fabs(M) >= 1.0) return 0.5 * (M + sgn * fabs(M));
    const double t = M * M - 1.0;
    return sgn * 0.25 * (M + sgn) * (M + sgn) + sgn * 0.125 * t * t;
}

static double ausm_pres(double M, int sgn)
{
    if (fabs(M) >= 1.0) return M * sgn > 0.0 ? 1.0 : 0.0;
    const double t = M * M - 1.0;
    return 0.25 * (M + sgn) * (M + sgn) * (2.0 - sgn * M) + sgn * 0.1875 * M * t * t;
}

static void ausm_plus(double g, int d, int k, const double* PL, const double* PR, const double* UL,
                      const double* UR, double* F)
{
    const int m = d + 2;
    const double pL = PL[d + 1], pR = PR[d + 1];
    const double HL = (UL[d + 1] + pL) / PL[0], HR = (UR[d + 1] + pR) / PR[0];
    const double uL = PL[1 + k], uR = PR[1 + k];
    const double asL = sqrt(2.0 * (g - 1.0) / (g + 1.0) * HL);
    const double asR = sqrt(2.0 * (g - 1.0) / (g + 1.0) * HR);
    const double atL = asL * asL / (asL > uL ? asL : uL);
    const double atR = asR * asR / (asR > -uR ? asR : -uR);
    const double a = atL < atR ? atL : atR;
    const double ML = uL / a, MR = uR / a;
    const double mh = ausm_mach(ML, 1) + ausm_mach(MR, -1);
    const double ph = ausm_pres(ML, 1) * pL + ausm_pres(MR, -1) * pR;
    const double mp = mh > 0.0 ? mh : 0.0, mm = mh < 0.0 ? mh : 0.0;
    double psiL[MMAX], psiR[MMAX];
    int v;
    psiL[0] = PL[0];
    psiR[0] = PR[0];
    for (v = 0; v < d; v++) {
        psiL[1 + v] = UL[1 + v];
        psiR[1 + v] = UR[1 + v];
    }
    psiL[d + 1] = PL[0] * HL;
    psiR[d + 1] = PR[0] * HR;
    for (v = 0; v < m; v++) F[v] = a * (mp * psiL[v] + mm * psiR[v]);
    F[1 + k] += ph;
}

/* numerical flux in direction k across the face between stencil cells 1 and 2
 * of W[0..3] (conservative values), face of width dxf. */
static void num_flux(Orc* o, int k, double dxf, double W[4][MMAX], double* F)
{
    int m = o->m, v;
    if (o->eq == 0) { /* linear advection, centred flux (Sec. 4.5) */
        double ak = o->cfg.phys[k];
        F[0] = ak * (W[1][0] + W[2][0]) / 2.0;
        return;
    }
    if (o->eq == 3) { /* reaction-diffusion: two-point diffusive flux */
        double D = o->cfg.phys[0];
        F[0] = -D * (W[2][0] - W[1][0]) / dxf;
        return;
    }
    if (o->eq == 1) { /* Burgers: MUSCL-minmod + Godunov for f = u^2/2 */
        double uL = W[1][0] + 0.5 * minmod(W[1][0] - W[0][0], W[2][0] - W[1][0]);
        double uR = W[2][0] - 0.5 * minmod(W[2][0] - W[1][0], W[3][0] - W[2][0]);
        double fL = 0.5 * uL * uL, fR = 0.5 * uR * uR;
        if (uL <= uR) {
            if (uL > 0.0) F[0] = fL;
            else if (uR < 0.0) F[0] = fR;
            else F[0] = 0.0;
        } else F[0] = fL > fR ? fL : fR;
        return;
    }
    /* Euler: MUSCL-minmod on primitive (rho, velocities, p), HLL flux */
    double g = o->cfg.phys[0];
    int d = o->d;
    double P[4][MMAX];
    int i;
    for (i = 0; i < 4; i++) {
        double rho = W[i][0], ke = 0.0;
        P[i][0] = rho;
        for (v = 0; v < d; v++) {
            P[i][1 + v] = W[i][1 + v] / rho;
            ke += W[i][1 + v] * P[i][1 + v];
        }
        P[i][d + 1] = (g - 1.0) * (W[i][d + 1] - 0.5 * ke);
    }
    double PL[MMAX], PR[MMAX], UL[MMAX], UR[MMAX], FL[MMAX], FR[MMAX];
    for (v = 0; v < m; v++) {
        PL[v] = P[1][v] + 0.5 * minmod(P[1][v] - P[0][v], P[2][v] - P[1][v]);
        PR[v] = P[2][v] - 0.5 * minmod(P[2][v] - P[1][v], P[3][v] - P[2][v]);
    }
    double keL = 0.0, keR = 0.0;
    UL[0] = PL[0];
    UR[0] = PR[0];
    for (v = 0; v < d; v++) {
        UL[1 + v] = PL[0] * PL[1 + v];
        UR[1 + v] = PR[0] * PR[1 + v];
        keL += PL[1 + v] * PL[1 + v];
        keR += PR[1 + v] * PR[1 + v];
    }
    UL[d + 1] = PL[d + 1] / (g - 1.0) + 0.5 * PL[0] * keL;
    UR[d + 1] = PR[d + 1] / (g - 1.0) + 0.5 * PR[0] * keR;
    double unL = PL[1 + k], unR = PR[1 + k];
    for (v = 0; v < m; v++) {
        FL[v] = UL[v] * unL;
        FR[v] = UR[v] * unR;
    }
    FL[1 + k] += PL[d + 1];
    FR[1 + k] += PR[d + 1];
    FL[d + 1] += PL[d + 1] * unL;
    FR[d + 1] += PR[d + 1] * unR;
    if (o->cfg.flux == 1) {
        ausm_plus(g, d, k, PL, PR, UL, UR, F);
        return;
    }
    double cL = sqrt(g * PL[d + 1] / PL[0]), cR = sqrt(g * PR[d + 1] / PR[0]);
    double sL = unL - cL < unR - cR ? unL - cL : unR - cR;
    double sR = unL + cL > unR + cR ? unL + cL : unR + cR;
    if (sL >= 0.0) {
        for (v = 0; v < m; v++) F[v] = FL[v];
    } else if (sR <= 0.0) {
        for (v = 0; v < m; v++) F[v] = FR[v];
    } else {
        for (v = 0; v < m; v++)
            F[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) / (sR - sL);
    }
}

/* point source S(q) (Sec. 2, below Eq. 2) */
static void source(Orc* o, const double* q, double* S)
{
    int v;
    for (v = 0; v < o->m; v++) S[v] = 0.0;
    if (o->eq == 3) {
        double k = o->cfg.phys[1], a = o->cfg.phys[2], u = q[0];
        S[0] = k * u * (1.0 - u) * (u - a);
    }
}

/* largest characteristic speed sum over directions, for the CFL step */
static double wave_speed(Orc* o, const double* q)
{
    int d = o->d, k;
    double s = 0.0;
    if (o->eq == 0) {
        for (k = 0; k < d; k++) s += fabs(o->cfg.phys[k]);
    } else if (o->eq == 1) {
        s = d * fabs(q[0]);
    } else if (o->eq == 2) {
        double g = o->cfg.phys[0], rho = q[0], ke = 0.0;
        for (k = 0; k < d; k++) ke += q[1 + k] * q[1 + k] / rho;
        double p = (g - 1.0) * (q[d + 1] - 0.5 * ke);
        double c = sqrt(g * p / rho);
        for (k = 0; k < d; k++) s += fabs(q[1 + k] / rho) + c;
    }
    return s;
}

/* ------------------------------------------------------------ fluxes */
enum { K_WALL = 0, K_LEAF = 1, K_FINER = 2, K_COARSER = 3 };

/* Face flux of the leaf at coords c of level u, direction k, side -1/+1,
 * oriented along +x_k.  Sec. 2 flux scenarios: with a same-level neighbour
 * (leaf or virtual) the flux is computed on level u; when the neighbour is
 * an internal node it is the mean of the 2^{d-1} sub-face fluxes computed on
 * level u+1 with the leaf's virtual children. */
static void face_flux(Orc* o, int u, const int c[3], int k, int side, const Ctx* x,
                      double* F, int* kind)
{
    int d = o->d, m = o->m, v, i, j;
    double W[4][MMAX];
    int nb[3] = {c[0], c[1], c[2]}, q;
    nb[k] += side;
    int sub = 0;
    if (!inside(o, u, k, nb[k], &q)) *kind = K_WALL;
    else {
        nb[k] = q;
        unsigned char s = o->st[u][lin(o, u, nb)];
        if (s == 2) sub = 1, *kind = K_FINER;
        else *kind = s == 1 ? K_LEAF : K_COARSER;
    }
    if (!sub) {
        int p[3] = {c[0], c[1], c[2]};
        int first = side > 0 ? c[k] - 1 : c[k] - 2;
        for (i = 0; i < 4; i++) {
            p[k] = first + i;
            value_at(o, u, p, x, W[i]);
        }
        num_flux(o, k, o->dx[u][k], W, F);
        return;
    }
    int ntan = 1 << (d - 1), t;
    double acc[MMAX], Fs[MMAX];
    for (v = 0; v < m; v++) acc[v] = 0.0;
    for (t = 0; t < ntan; t++) {
        int p[3] = {0, 0, 0}, bit = 0;
        for (j = 0; j < d; j++) {
            if (j == k) continue;
            p[j] = 2 * c[j] + ((t >> bit) & 1);
            bit++;
        }
        int first = side > 0 ? 2 * c[k] : 2 * c[k] - 2;
        for (i = 0; i < 4; i++) {
            p[k] = first + i;
            value_at(o, u + 1, p, x, W[i]);
        }
        num_flux(o, k, o->dx[u + 1][k], W, Fs);
        for (v = 0; v < m; v++) acc[v] += Fs[v];
    }
    for (v = 0; v < m; v++) F[v] = acc[v] / ntan;
}

/* right-hand side f of the leaf (Eq. 2): -sum_k (F_{k,+} - F_{k,-}) / dx + S */
static void leaf_rhs(Orc* o, int u, long id, const Ctx* x, double* f,
                     double Fr[6][MMAX], int kinds[6])
{
    int d = o->d, m = o->m, k, v, c[3];
    double self[MMAX], Fm[MMAX], Fp[MMAX];
    coords(o, u, id, c);
    expose(o, u, id, x, self);
    source(o, self, f);
    for (k = 0; k < d; k++) {
        face_flux(o, u, c, k, -1, x, Fm, &kinds[2 * k]);
        face_flux(o, u, c, k, +1, x, Fp, &kinds[2 * k + 1]);
        for (v = 0; v < m; v++) {
            Fr[2 * k][v] = Fm[v];
            Fr[2 * k + 1][v] = Fp[v];
            f[v] += (Fm[v] - Fp[v]) / o->dx[u][k];
        }
    }
}

/* flux registers (extension; the paper is silent on conservation across
 * levels): each coarse-fine face accumulates the time-integrated flux seen by
 * the coarse leaf (RC) and by each fine leaf (RF), weight dt_l * b_s. */
static void reg_add(Orc* o, int u, long id, double w, double Fr[6][MMAX], const int kinds[6])
{
    int m = o->m, fi, v;
    if (o->gts || !o->cfg.reflux) return;
    for (fi = 0; fi < o->nf; fi++) {
        double* R = NULL;
        if (kinds[fi] == K_FINER) R = o->RC[u] + ((long)id * o->nf + fi) * m;
        else if (kinds[fi] == K_COARSER) R = o->RF[u] + ((long)id * o->nf + fi) * m;
        if (!R) continue;
        for (v = 0; v < m; v++) R[v] += w * Fr[fi][v];
    }
}

/* ------------------------------------------------------------ projections */
static int nchild(const Orc* o) { return 1 << o->d; }

static long child_id(const Orc* o, int l, const int c[3], int t)
{
    int p[3] = {0, 0, 0}, k;
    for (k = 0; k < o->d; k++) p[k] = 2 * c[k] + ((t >> k) & 1);
    return lin(o, l + 1, p);
}

/* projection P_{l+1 -> l}: mean of the children (Eq. 3) of field src into
 * field dst, for every internal node of level l */
static void project_mean(Orc* o, int l, double** src, double** dst)
{
    int m = o->m, v, t, c[3], nch = nchild(o);
    long id;
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        coords(o, l, id, c);
        double acc[MMAX] = {0};
        for (t = 0; t < nch; t++) {
            const double* s = V(src, l + 1, child_id(o, l, c, t));
            for (v = 0; v < m; v++) acc[v] += s[v];
        }
        double* D = V(dst, l, id);
        for (v = 0; v < m; v++) D[v] = acc[v] / nch;
    }
}

/* Value of node (l, id) at t^n + 2 dt_l, extrapolated from its own stage
 * values: a leaf's Eq. 14 value q* + k2 (stored as QX by its second stage), an
 * internal node's Eq. 15 value 2 q* - q^n (its q* is the projected value at
 * t^n + dt_l). */
static void value_two_steps(Orc* o, int l, long id, double* out)
{
    int v;
    if (o->st[l][id] == 1) {
        memcpy(out, V(o->QX, l, id), sizeof(double) * o->m);
        return;
    }
    const double* s1 = V(o->Q1, l, id);
    const double* s0 = V(o->Q0, l, id);
    for (v = 0; v < o->m; v++) out[v] = 2.0 * s1[v] - s0[v];
}

/* q* of the internal nodes of level l for the second stage of their level:
 * their value at t^n + dt_l = t^n + 2 dt_{l+1}, the mean (Eq. 3) of the
 * children's values at that instant (Eqs. 14-15); this is Alg. 4. */
static void project_rk2(Orc* o, int l)
{
    int m = o->m, v, t, c[3], nch = nchild(o);
    long id;
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        coords(o, l, id, c);
        double acc[MMAX] = {0}, w[MMAX];
        for (t = 0; t < nch; t++) {
            value_two_steps(o, l + 1, child_id(o, l, c, t), w);
            for (v = 0; v < m; v++) acc[v] += w[v];
        }
        double* D = V(o->Q1, l, id);
        for (v = 0; v < m; v++) D[v] = acc[v] / nch;
    }
}

/* Stage-3 values of the internal nodes of level l (Alg. 6): q** is their
 * value at t^n + dt_{l+1}, the mean (Eq. 3) of the children's end values
 * (every child, leaf or internal, ends its first sub-step there), and the end
 * value at t^n + dt_l follows from Eq. 16 (READING: with the theta values
 * implied by the projected q**, Eq. 16 reduces to 2 q** - q^n). */
static void project_rk3(Orc* o, int l)
{
    int m = o->m, v;
    long id;
    project_mean(o, l, o->QE, o->Q2);
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        const double* q2 = V(o->Q2, l, id);
        const double* q0 = V(o->Q0, l, id);
        double* qe = V(o->QE, l, id);
        for (v = 0; v < m; v++) qe[v] = 2.0 * q2[v] - q0[v];
    }
}

/* Alg. 8: tree refreshing before the second RK step -- half-step value of an
 * internal node = mean of its children's q* (Eq. 17), then q* by Eq. 18 */
static void refresh_rk2(Orc* o, int l)
{
    int m = o->m, v;
    long id;
    project_mean(o, l, o->Q1, o->XH);
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        double* q1 = V(o->Q1, l, id);
        const double* xh = V(o->XH, l, id);
        const double* q0 = V(o->Q0, l, id);
        for (v = 0; v < m; v++) q1[v] = 2.0 * xh[v] - q0[v];
    }
}

/* Alg. 9: tree refreshing before the third RK step -- theta=1/4 value of an
 * internal node = mean of its children's q**, then Eq. 20 (theta=3/4) and
 * Eq. 21 (q**), with q* the node's latest stored value (READING: the Alg. 4
 * overwrite) */
static void refresh_rk3(Orc* o, int l)
{
    int m = o->m, v;
    long id;
    project_mean(o, l, o->Q2, o->N1);
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        const double* q0 = V(o->Q0, l, id);
        const double* q1 = V(o->Q1, l, id);
        const double* n1 = V(o->N1, l, id);
        double* n3 = V(o->N3, l, id);
        double* q2 = V(o->Q2, l, id);
        for (v = 0; v < m; v++) {
            n3[v] = -13.0 / 2.0 * q0[v] - 3.0 / 2.0 * q1[v] + 9.0 * n1[v];
            q2[v] = -11.0 / 2.0 * q0[v] - 3.0 / 2.0 * q1[v] + 8.0 * n1[v];
        }
    }
}

/* Alg. 3 (first block) and Sec. 4.3: internal nodes of the mid-step level
 * lmin-1 take the projection of their children (now at t^n = theta 1/2 of
 * their own step) as their theta=1/2 value (RK2) or q** (RK3), and the end
 * value at t^n + dt_lmin by Eq. 22 (RK2) or 2 q** - q^n (RK3, Eq. 16 with
 * the implied theta values).  RK3 also rebuilds theta=1/4, 3/4 from Eqs.
 * 20, 21 for the third stage of level lmin (Alg. 9, l = lmin branch). */
static void refresh_mid(Orc* o, int l)
{
    int m = o->m, v;
    long id;
    if (o->rk == 2) project_mean(o, l, o->Q0, o->NH);
    else project_mean(o, l, o->Q0, o->Q2);
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 2) continue;
        const double* q0 = V(o->Q0, l, id);
        const double* q1 = V(o->Q1, l, id);
        double* qe = V(o->QE, l, id);
        if (o->rk == 2) {
            const double* nh = V(o->NH, l, id);
            for (v = 0; v < m; v++) qe[v] = -2.0 * q0[v] - q1[v] + 4.0 * nh[v];
        } else {
            const double* q2 = V(o->Q2, l, id);
            double* n1 = V(o->N1, l, id);
            double* n3 = V(o->N3, l, id);
            for (v = 0; v < m; v++) {
                qe[v] = 2.0 * q2[v] - q0[v];
                n1[v] = (q2[v] + 11.0 / 2.0 * q0[v] + 3.0 / 2.0 * q1[v]) / 8.0;
                n3[v] = -13.0 / 2.0 * q0[v] - 3.0 / 2.0 * q1[v] + 9.0 * n1[v];
            }
        }
    }
}

/* ------------------------------------------------------------ adaptation */
static double eps_level(const Orc* o, int l)
{
    if (o->cfg.eps_mode == 1) return ldexp(o->cfg.eps, o->d * (l - o->L));
    return o->cfg.eps;
}

/* detail norm of an internal node (Eq. 5): max over children and variables of
 * |q_child - predicted_child| / s_v, s_v the largest |q_v| over leaves at the
 * last full adaptation (READING: the paper does not fix the norm) */
static double detail_norm(Orc* o, int l, long id)
{
    int m = o->m, v, t, c[3], nch = nchild(o), k;
    Ctx x = {l, 0, o->lb};
    double qt[MMAX], nrm = 0.0;
    coords(o, l, id, c);
    for (t = 0; t < nch; t++) {
        int p[3] = {0, 0, 0};
        for (k = 0; k < o->d; k++) p[k] = 2 * c[k] + ((t >> k) & 1);
        predict_cell(o, l + 1, p, &x, qt);
        const double* q = V(o->Q0, l + 1, lin(o, l + 1, p));
        for (v = 0; v < m; v++) {
            double a = fabs(q[v] - qt[v]) / o->scale[v];
            if (a > nrm) nrm = a;
        }
    }
    return nrm;
}

static void update_scale(Orc* o)
{
    int v, l;
    long id;
    for (v = 0; v < o->m; v++) o->scale[v] = 1e-14;
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++) {
            if (o->st[l][id] != 1) continue;
            const double* q = V(o->Q0, l, id);
            for (v = 0; v < o->m; v++)
                if (fabs(q[v]) > o->scale[v]) o->scale[v] = fabs(q[v]);
        }
}

/* iterate over the 3^d offsets within Chebyshev radius 1 */
#define FOR_NEIGH(o, OFF)                                         \
    for (int _z = ((o)->d > 2 ? -1 : 0); _z <= ((o)->d > 2 ? 1 : 0); _z++) \
        for (int _y = ((o)->d > 1 ? -1 : 0); _y <= ((o)->d > 1 ? 1 : 0); _y++) \
            for (int _x = -1; _x <= 1; _x++)                      \
                for (int OFF[3] = {_x, _y, _z}, _once = 1; _once; _once = 0)

/* map c+off at level l through the tree-neighbourhood rule */
static int nb_id(const Orc* o, int l, const int c[3], const int off[3], long* id)
{
    int p[3] = {0, 0, 0}, k;
    for (k = 0; k < o->d; k++)
        if (!inside(o, l, k, c[k] + off[k], &p[k])) return 0;
    *id = lin(o, l, p);
    return 1;
}

/* Install a new refinement map Rn (levels la..L-1; Rn[l][i] = node i of level
 * l has children) and carry the values over: kept nodes keep theirs, new
 * nodes are predicted from their parent level top-down (Sec. 2), merged
 * nodes already hold the projection of their children. */
static void apply_tree(Orc* o, int la, unsigned char** Rn)
{
    int L = o->L, m = o->m, l, v, c[3];
    long id;
    Ctx x0 = {la, 0, o->lb};
    for (l = la; l <= L; l++) {
        unsigned char* old = (unsigned char*)malloc(o->nc[l]);
        memcpy(old, o->st[l], o->nc[l]);
        for (id = 0; id < o->nc[l]; id++) {
            int exists;
            coords(o, l, id, c);
            if (l == la) exists = o->st[l][id] != 0;
            else {
                int p[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
                exists = Rn[l - 1][lin(o, l - 1, p)] != 0;
            }
            int refined = l < L && Rn[l][id];
            if (refined && !exists) fail(o, "apply_tree: refined node without parent");
            o->st[l][id] = exists ? (refined ? 2 : 1) : 0;
        }
        for (id = 0; id < o->nc[l]; id++) {
            unsigned char s = o->st[l][id];
            if (s == old[id]) continue;
            if (s != 0 && old[id] == 0) {
                coords(o, l, id, c);
                predict_cell(o, l, c, &x0, V(o->Q0, l, id));
            }
            if (s == 1) memcpy(V(o->QE, l, id), V(o->Q0, l, id), sizeof(double) * m);
            if (o->RC[l]) {
                for (v = 0; v < o->nf * m; v++) {
                    o->RC[l][id * o->nf * m + v] = 0.0;
                    o->RF[l][id * o->nf * m + v] = 0.0;
                }
            }
        }
        free(old);
    }
    /* projection of the new internal nodes, bottom-up (Eq. 3) */
    for (l = L - 1; l >= la; l--) project_mean(o, l, o->Q0, o->Q0);
}

/* Alg. 1 + Alg. 2 with the graded-tree rules, restricted to levels >= la
 * (Sec. 4 "Adapting the grid during local time-stepping": only levels that
 * share the current instant may split or merge).  READINGS:
 *  - a node of level l keeps its children iff its detail norm > eps_{l+1};
 *  - space safety: the 3^d neighbours of a significant node are refined too;
 *  - scale safety: if the norm exceeds 8 eps_{l+1} its children are refined;
 *  - grading: refining (l,i) requires refining every (l-1, floor(i/2)+delta),
 *    |delta|_inf <= 1, which gives every leaf a radius-2 same-level stencil
 *    whose virtual cells are predicted from stored parent-level nodes;
 *  - at a partial remesh, refinements that would need a change below la are
 *    dropped ("Allowed" mask computed top-down from the frozen level la-1);
 *  - eps = 0 means no coarsening (uniform level L). */
static void adapt(Orc* o, int la)
{
    int L = o->L, l, t;
    long id;
    int c[3];
    if (la >= L) return;
    if (la == o->lb) update_scale(o);
    unsigned char *D[LMAX + 1] = {0}, *A[LMAX + 1] = {0}, *S[LMAX + 1] = {0}, *B[LMAX + 1] = {0};
    for (l = la; l < L; l++) {
        D[l] = (unsigned char*)calloc(o->nc[l], 1);
        A[l] = (unsigned char*)calloc(o->nc[l], 1);
        S[l] = (unsigned char*)calloc(o->nc[l], 1);
        B[l] = (unsigned char*)calloc(o->nc[l], 1);
    }
    /* 1. details and significance (Alg. 2 inner comparison) */
    for (l = la; l < L; l++) {
        double el = eps_level(o, l + 1);
        for (id = 0; id < o->nc[l]; id++) {
            if (o->st[l][id] != 2) continue;
            if (o->cfg.eps <= 0.0) {
                S[l][id] = 1;
                continue;
            }
            double nrm = detail_norm(o, l, id);
            if (fabs(nrm - el) <= 1e-10 * el || fabs(nrm - 8.0 * el) <= 8e-10 * el) o->near++;
            S[l][id] = nrm > el;
            B[l][id] = nrm > 8.0 * el;
        }
    }
    /* 2. desired refinement: significance, space safety, scale safety */
    for (l = la; l < L; l++) {
        for (id = 0; id < o->nc[l]; id++) {
            if (o->cfg.eps <= 0.0) {
                D[l][id] = 1;
                continue;
            }
            if (!S[l][id]) continue;
            coords(o, l, id, c);
            FOR_NEIGH(o, off)
            {
                long j;
                if (nb_id(o, l, c, off, &j)) D[l][j] = 1;
            }
            if (B[l][id] && l + 1 < L)
                for (t = 0; t < nchild(o); t++) D[l + 1][child_id(o, l, c, t)] = 1;
        }
    }
    /* 3. admissible refinements, top-down from the frozen level la-1 */
    for (l = la; l < L; l++) {
        for (id = 0; id < o->nc[l]; id++) {
            if (la == o->lb && l == la) {
                A[l][id] = 1;
                continue;
            }
            coords(o, l, id, c);
            int P[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1}, ok = 1;
            FOR_NEIGH(o, off)
            {
                long j;
                if (!nb_id(o, l - 1, P, off, &j)) continue;
                if (l - 1 < la) ok &= o->st[l - 1][j] == 2;
                else ok &= A[l - 1][j];
            }
            A[l][id] = (unsigned char)ok;
        }
    }
    /* 4. closure, fine to coarse */
    for (l = la; l < L; l++)
        for (id = 0; id < o->nc[l]; id++) D[l][id] = D[l][id] && A[l][id];
    for (l = L - 1; l > la; l--) {
        for (id = 0; id < o->nc[l]; id++) {
            if (!D[l][id]) continue;
            coords(o, l, id, c);
            int P[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
            FOR_NEIGH(o, off)
            {
                long j;
                if (nb_id(o, l - 1, P, off, &j)) D[l - 1][j] = 1;
            }
        }
    }
    apply_tree(o, la, D);
    for (l = la; l < L; l++) {
        free(D[l]);
        free(A[l]);
        free(S[l]);
        free(B[l]);
    }
}

/* ------------------------------------------------------------ time stepping */
static int level_min(const Orc* o, long long n)
{
    int l;
    for (l = o->lb; l <= o->L; l++)
        if (n % (1LL << (o->L - l)) == 0) return l;
    return o->L;
}

static const double RK_B2[2] = {0.5, 0.5};
static const double RK_B3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};

static double bweight(const Orc* o, int s) { return o->rk == 2 ? RK_B2[s - 1] : RK_B3[s - 1]; }

/* one compact RK stage (Sec. 3) on every leaf of level u; dtl = step of the
 * level; the NERK partial sums are formed right after each stage as the
 * paper stores them (Eq. 12 and the theta = 1/4, 3/4 rules). */
static void stage_level(Orc* o, int u, int s, int lmin, double dtl)
{
    int m = o->m, v;
    long id;
    Ctx x = {u, s, lmin};
    double f[MMAX], Fr[6][MMAX];
    int kinds[6];
    for (id = 0; id < o->nc[u]; id++) {
        if (o->st[u][id] != 1) continue;
        leaf_rhs(o, u, id, &x, f, Fr, kinds);
        double* q0 = V(o->Q0, u, id);
        double* q1 = V(o->Q1, u, id);
        double* q2 = V(o->Q2, u, id);
        double* qe = V(o->QE, u, id);
        double* nh = V(o->NH, u, id);
        double* n1 = V(o->N1, u, id);
        double* n3 = V(o->N3, u, id);
        double* qx = V(o->QX, u, id);
        for (v = 0; v < m; v++) {
            double kk = dtl * f[v];
            if (s == 1) {
                q1[v] = q0[v] + kk;
                if (o->rk == 2) nh[v] = q0[v] + 3.0 / 8.0 * kk;
                else {
                    n1[v] = q0[v] + 7.0 / 32.0 * kk;
                    n3[v] = q0[v] + 15.0 / 32.0 * kk;
                }
            } else if (s == 2) {
                qx[v] = q1[v] + kk; /* Eq. 14 */
                if (o->rk == 2) {
                    qe[v] = 0.5 * q0[v] + 0.5 * q1[v] + 0.5 * kk;
                    nh[v] = nh[v] + 1.0 / 8.0 * kk;
                } else {
                    q2[v] = 0.75 * q0[v] + 0.25 * q1[v] + 0.25 * kk;
                    n1[v] = n1[v] + 1.0 / 32.0 * kk;
                    n3[v] = n3[v] + 9.0 / 32.0 * kk;
                }
            } else {
                qe[v] = 1.0 / 3.0 * q0[v] + 2.0 / 3.0 * q2[v] + 2.0 / 3.0 * kk;
            }
        }
        reg_add(o, u, id, dtl * bweight(o, s), Fr, kinds);
        if (s == 1) o->updates++;
    }
}

/* conservative correction of the coarse leaves of level l whose step has just
 * ended: q_c += +-(coarse register - mean of the fine registers) / dx */
static void reflux_level(Orc* o, int l)
{
    int d = o->d, m = o->m, k, v, j, c[3], fi, t;
    long id;
    for (id = 0; id < o->nc[l]; id++) {
        if (o->st[l][id] != 1) continue;
        coords(o, l, id, c);
        for (fi = 0; fi < o->nf; fi++) {
            k = fi / 2;
            int side = (fi & 1) ? 1 : -1, q;
            int nb[3] = {c[0], c[1], c[2]};
            if (!inside(o, l, k, c[k] + side, &q)) continue;
            nb[k] = q;
            if (o->st[l][lin(o, l, nb)] != 2) continue;
            int ntan = 1 << (d - 1), opp = 2 * k + (side > 0 ? 0 : 1);
            double g[MMAX] = {0};
            for (t = 0; t < ntan; t++) {
                int p[3] = {0, 0, 0}, bit = 0;
                for (j = 0; j < d; j++) {
                    if (j == k) continue;
                    p[j] = 2 * nb[j] + ((t >> bit) & 1);
                    bit++;
                }
                p[k] = 2 * nb[k] + (side > 0 ? 0 : 1);
                long ch = lin(o, l + 1, p);
                if (o->st[l + 1][ch] != 1) fail(o, "reflux: fine cell is not a leaf");
                const double* rf = o->RF[l + 1] + ((long)ch * o->nf + opp) * m;
                for (v = 0; v < m; v++) g[v] += rf[v];
            }
            const double* rc = o->RC[l] + ((long)id * o->nf + fi) * m;
            double* qe = V(o->QE, l, id);
            for (v = 0; v < m; v++)
                qe[v] += side * (rc[v] - g[v] / ntan) / o->dx[l][k];
        }
    }
}

static void begin_step(Orc* o, int lmin)
{
    int l;
    long id;
    for (l = lmin; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) memcpy(V(o->Q0, l, id), V(o->QE, l, id), sizeof(double) * o->m);
    for (l = o->L - 1; l >= lmin; l--) project_mean(o, l, o->Q0, o->Q0);
}

/* Alg. 3: one iteration n (0-based within the macro step) of the LT scheme */
static void lt_iteration(Orc* o, long long n, long long nit)
{
    int L = o->L, lb = o->lb, l;
    int lmin = level_min(o, n);
    double dt = o->dt;
    begin_step(o, lmin);
    if (o->cfg.adapt_mode == 2 || (o->cfg.adapt_mode == 1 && n == 0)) adapt(o, lmin);
    if (lmin > lb) refresh_mid(o, lmin - 1);
    /* first RK step on every active level */
    for (l = L; l >= lmin; l--) stage_level(o, l, 1, lmin, ldexp(dt, L - l));
    /* Alg. 8 then Alg. 5 */
    for (l = L - 1; l >= lmin; l--) refresh_rk2(o, l);
    for (l = L; l >= lmin; l--) {
        if (l < L) project_rk2(o, l);
        stage_level(o, l, 2, lmin, ldexp(dt, L - l));
    }
    if (o->rk == 3) { /* Alg. 9 then Alg. 7 */
        for (l = L - 1; l >= lmin; l--) refresh_rk3(o, l);
        for (l = L; l >= lmin; l--) {
            if (l < L) project_rk3(o, l);
            stage_level(o, l, 3, lmin, ldexp(dt, L - l));
        }
    }
    /* levels whose step ends with this iteration: apply and clear registers */
    if (o->cfg.reflux) {
        int lc = (n + 1 == nit) ? lb : level_min(o, n + 1);
        for (l = lc; l < L; l++) reflux_level(o, l);
        for (l = lc; l <= L; l++) {
            memset(o->RC[l], 0, sizeof(double) * o->nc[l] * o->nf * o->m);
            if (l > lc) memset(o->RF[l], 0, sizeof(double) * o->nc[l] * o->nf * o->m);
        }
    }
}

/* MR with one global time step (MR/RK2, MR/RK3): every leaf advances with
 * the finest-level step; internal nodes are plain projections of the stage
 * values, virtual cells predictions at the same instant. */
static void gts_iteration(Orc* o, long long n)
{
    int L = o->L, lb = o->lb, l;
    double dt = o->dt;
    begin_step(o, lb);
    if (o->cfg.adapt_mode == 2 || (o->cfg.adapt_mode == 1 && n == 0)) adapt(o, lb);
    for (l = L; l >= lb; l--) stage_level(o, l, 1, lb, dt);
    for (l = L - 1; l >= lb; l--) project_mean(o, l, o->Q1, o->Q1);
    for (l = L; l >= lb; l--) stage_level(o, l, 2, lb, dt);
    if (o->rk == 3) {
        for (l = L - 1; l >= lb; l--) project_mean(o, l, o->Q2, o->Q2);
        for (l = L; l >= lb; l--) stage_level(o, l, 3, lb, dt);
    }
}

static int check_finite(Orc* o)
{
    int l, v;
    long id;
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++) {
            if (o->st[l][id] != 1) continue;
            const double* q = V(o->QE, l, id);
            for (v = 0; v < o->m; v++)
                if (!isfinite(q[v])) {
                    fail(o, "non-finite value at level %d cell %ld", l, id);
                    return OR_E_NUMERIC;
                }
        }
    return OR_OK;
}

/* run n fine iterations with step dt (dt may only change at a macro-step
 * boundary, where every level is at the same instant) */
static int run_iters(Orc* o, double dt, long long n)
{
    long long nit = 1LL << (o->L - o->lb), i;
    if (o->pos != 0 && dt != o->dt) {
        fail(o, "dt changed inside a macro step");
        return OR_E_STATE;
    }
    o->dt = dt;
    for (i = 0; i < n; i++) {
        if (o->gts) gts_iteration(o, o->pos);
        else lt_iteration(o, o->pos, nit);
        o->iters++;
        o->pos++;
        if (o->bad) return OR_E_STATE;
        if (o->pos == nit) {
            o->pos = 0;
            o->macros++;
            int r = check_finite(o);
            if (r) return r;
        }
    }
    return OR_OK;
}

/* CFL step of the finest level (READING of Eq. 13 and the Courant number
 * sigma of Sec. 5): dt = sigma * min(dx_L / max_leaves sum_k lambda_k,
 * dx_L^2 / (2 d D)) */
static double cfl_dt(Orc* o)
{
    int l;
    long id;
    double lam = 0.0, dxm = o->dx[o->L][0];
    for (l = 1; l < o->d; l++)
        if (o->dx[o->L][l] < dxm) dxm = o->dx[o->L][l];
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) {
                double s = wave_speed(o, V(o->QE, l, id));
                if (s > lam) lam = s;
            }
    double dt = lam > 0.0 ? dxm / lam : dxm;
    if (o->eq == 3) {
        double dd = dxm * dxm / (2.0 * o->d * o->cfg.phys[0]);
        if (lam <= 0.0 || dd < dt) dt = dd;
    }
    return o->cfg.cfl * dt;
}

/* ------------------------------------------------------------ API */
static void free_all(Orc* o)
{
    int l;
    for (l = 0; l <= LMAX; l++) {
        free(o->st[l]);
        free(o->Q0[l]);
        free(o->Q1[l]);
        free(o->Q2[l]);
        free(o->QE[l]);
        free(o->XH[l]);
        free(o->NH[l]);
        free(o->N1[l]);
        free(o->N3[l]);
        free(o->QX[l]);
        free(o->RC[l]);
        free(o->RF[l]);
    }
}

int or_create(const or_config* cfg, const double* q0, void** out)
{
    *out = NULL;
    if (!cfg || !q0) return OR_E_INVALID;
    if (cfg->dim < 1 || cfg->dim > 3 || cfg->max_level < 1 || cfg->max_level > LMAX ||
        cfg->min_level < 0 || cfg->min_level > cfg->max_level || cfg->equation < 0 ||
        cfg->equation > 3 || (cfg->rk_order != 2 && cfg->rk_order != 3) ||
        cfg->precision != 0 || cfg->time_mode < 0 || cfg->time_mode > 1 ||
        cfg->dim * cfg->max_level > 30 || cfg->flux < 0 || cfg->flux > 1 ||
        (cfg->flux == 1 && cfg->equation != 2))
        return OR_E_INVALID;
    {
        int k;
        for (k = 0; k < cfg->dim; k++)
            if (cfg->bc[k] < 0 || cfg->bc[k] > 2 || (cfg->bc[k] == 2 && cfg->equation == 2))
                return OR_E_INVALID; /* zero Dirichlet: scalar equations only */
    }
    Orc* o = (Orc*)calloc(1, sizeof(Orc));
    if (!o) return OR_E_NOMEM;
    o->cfg = *cfg;
    o->d = cfg->dim;
    o->m = cfg->equation == 2 ? cfg->dim + 2 : 1;
    o->L = cfg->max_level;
    o->lb = cfg->min_level;
    o->eq = cfg->equation;
    o->rk = cfg->rk_order;
    o->gts = cfg->time_mode == 0;
    o->nf = 2 * o->d;
    int l, k, m = o->m, v;
    long id;
    for (l = o->lb; l <= o->L; l++) {
        o->n[l] = 1 << l;
        o->nc[l] = 1L << (o->d * l);
        o->vol[l] = 1.0;
        for (k = 0; k < 3; k++) {
            o->dx[l][k] = (cfg->hi[k] - cfg->lo[k]) / o->n[l];
            if (k < o->d) o->vol[l] *= o->dx[l][k];
        }
        size_t nv = (size_t)o->nc[l] * m;
        o->st[l] = (unsigned char*)calloc(o->nc[l], 1);
        o->Q0[l] = (double*)calloc(nv, sizeof(double));
        o->Q1[l] = (double*)calloc(nv, sizeof(double));
        o->Q2[l] = (double*)calloc(nv, sizeof(double));
        o->QE[l] = (double*)calloc(nv, sizeof(double));
        o->XH[l] = (double*)calloc(nv, sizeof(double));
        o->NH[l] = (double*)calloc(nv, sizeof(double));
        o->N1[l] = (double*)calloc(nv, sizeof(double));
        o->N3[l] = (double*)calloc(nv, sizeof(double));
        o->QX[l] = (double*)calloc(nv, sizeof(double));
        if (cfg->reflux && !o->gts) {
            o->RC[l] = (double*)calloc(nv * o->nf, sizeof(double));
            o->RF[l] = (double*)calloc(nv * o->nf, sizeof(double));
        }
        if (!o->st[l] || !o->Q0[l] || !o->Q1[l] || !o->Q2[l] || !o->QE[l] || !o->XH[l] ||
            !o->NH[l] || !o->N1[l] || !o->N3[l] || !o->QX[l] ||
            (cfg->reflux && !o->gts && (!o->RC[l] || !o->RF[l]))) {
            free_all(o);
            free(o);
            return OR_E_NOMEM;
        }
        for (id = 0; id < o->nc[l]; id++) o->st[l][id] = l < o->L ? 2 : 1;
    }
    /* finest-level cell averages, input layout [var][cell] */
    for (id = 0; id < o->nc[o->L]; id++)
        for (v = 0; v < m; v++) o->Q0[o->L][id * m + v] = q0[(long)v * o->nc[o->L] + id];
    for (l = o->L - 1; l >= o->lb; l--) project_mean(o, l, o->Q0, o->Q0);
    update_scale(o);
    if (cfg->adapt_mode != 0) adapt(o, o->lb);
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) memcpy(V(o->QE, l, id), V(o->Q0, l, id), sizeof(double) * m);
    if (o->bad) {
        int r = OR_E_STATE;
        fprintf(stderr, "or_create: %s\n", o->err);
        free_all(o);
        free(o);
        return r;
    }
    *out = o;
    return OR_OK;
}

int or_set_tree(void* h, const unsigned char* lev)
{
    Orc* o = (Orc*)h;
    int L = o->L, lb = o->lb, l, c[3], k;
    long id;
    if (!o || !lev) return OR_E_INVALID;
    unsigned char* R[LMAX + 1] = {0};
    for (l = lb; l <= L; l++) R[l] = (unsigned char*)calloc(o->nc[l], 1);
    for (id = 0; id < o->nc[L]; id++) {
        if (lev[id] < lb || lev[id] > L) {
            snprintf(o->err, sizeof o->err, "set_tree: level out of range");
            for (l = lb; l <= L; l++) free(R[l]);
            return OR_E_INVALID;
        }
        coords(o, L, id, c);
        for (l = lb; l < lev[id]; l++) {
            int p[3] = {0, 0, 0};
            for (k = 0; k < o->d; k++) p[k] = c[k] >> (L - l);
            R[l][lin(o, l, p)] = 1;
        }
    }
    int ok = 1;
    for (id = 0; id < o->nc[L] && ok; id++) { /* every finest cell lies in a leaf of its level */
        coords(o, L, id, c);
        int lv = lb;
        for (l = lb; l < L; l++) {
            int p[3] = {0, 0, 0};
            for (k = 0; k < o->d; k++) p[k] = c[k] >> (L - l);
            if (!R[l][lin(o, l, p)]) break;
            lv = l + 1;
        }
        if (lv != lev[id]) ok = 0;
    }
    for (l = L - 1; l > lb && ok; l--) /* graded */
        for (id = 0; id < o->nc[l] && ok; id++) {
            if (!R[l][id]) continue;
            coords(o, l, id, c);
            int P[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
            FOR_NEIGH(o, off)
            {
                long j;
                if (nb_id(o, l - 1, P, off, &j) && !R[l - 1][j]) ok = 0;
            }
        }
    if (!ok) {
        snprintf(o->err, sizeof o->err, "set_tree: map is not a graded leaf partition");
        for (l = lb; l <= L; l++) free(R[l]);
        return OR_E_INVALID;
    }
    for (l = lb; l <= L; l++)
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) memcpy(V(o->Q0, l, id), V(o->QE, l, id), sizeof(double) * o->m);
    for (l = L - 1; l >= lb; l--) project_mean(o, l, o->Q0, o->Q0);
    apply_tree(o, lb, R);
    for (l = lb; l <= L; l++) {
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) memcpy(V(o->QE, l, id), V(o->Q0, l, id), sizeof(double) * o->m);
        free(R[l]);
    }
    return o->bad ? OR_E_STATE : OR_OK;
}

int or_adapt(void* h)
{
    Orc* o = (Orc*)h;
    int l;
    long id;
    if (!o) return OR_E_INVALID;
    begin_step(o, o->lb);
    adapt(o, o->lb);
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++)
            if (o->st[l][id] == 1) memcpy(V(o->QE, l, id), V(o->Q0, l, id), sizeof(double) * o->m);
    return o->bad ? OR_E_STATE : OR_OK;
}

int or_step(void* h, double t_target, long long* iters_out)
{
    Orc* o = (Orc*)h;
    if (!o) return OR_E_INVALID;
    if (o->pos != 0) return OR_E_STATE;
    long long it0 = o->iters, nit = 1LL << (o->L - o->lb);
    while (o->t < t_target) {
        double dt = cfl_dt(o);
        int last = 0;
        if (o->t + nit * dt >= t_target * (1.0 - 1e-14)) {
            dt = (t_target - o->t) / nit;
            last = 1;
        }
        double t0 = o->t;
        int r = run_iters(o, dt, nit);
        if (r) return r;
        o->t = last ? t_target : t0 + nit * dt;
    }
    if (iters_out) *iters_out = o->iters - it0;
    return OR_OK;
}

int or_iterate(void* h, double dt, long long n_iters, long long* iters_out)
{
    Orc* o = (Orc*)h;
    if (!o || !(dt > 0.0) || n_iters < 0) return OR_E_INVALID;
    long long it0 = o->iters, i;
    for (i = 0; i < n_iters; i++) {
        int r = run_iters(o, dt, 1);
        if (r) return r;
        o->t += dt;
    }
    if (iters_out) *iters_out = o->iters - it0;
    return OR_OK;
}

/* inverse MR transform of the synchronised leaves onto level L (Sec. 1:
 * the adapted grid rebuilt on a regular grid): internal nodes are projected
 * bottom-up, absent cells predicted top-down level by level. */
static void uniform(Orc* o, double* out)
{
    int L = o->L, lb = o->lb, m = o->m, l, v, c[3];
    long id;
    double* T[LMAX + 1] = {0};
    for (l = lb; l <= L; l++) T[l] = (double*)calloc((size_t)o->nc[l] * m, sizeof(double));
    for (l = L; l >= lb; l--)
        for (id = 0; id < o->nc[l]; id++) {
            if (o->st[l][id] == 1) memcpy(T[l] + id * m, V(o->QE, l, id), sizeof(double) * m);
            else if (o->st[l][id] == 2) {
                int t, nch = nchild(o);
                double acc[MMAX] = {0};
                coords(o, l, id, c);
                for (t = 0; t < nch; t++) {
                    const double* s = T[l + 1] + child_id(o, l, c, t) * m;
                    for (v = 0; v < m; v++) acc[v] += s[v];
                }
                for (v = 0; v < m; v++) T[l][id * m + v] = acc[v] / nch;
            }
        }
    /* top-down prediction into absent cells, using a temporary full status */
    unsigned char* keep[LMAX + 1];
    for (l = lb; l <= L; l++) {
        keep[l] = o->st[l];
        o->st[l] = (unsigned char*)malloc(o->nc[l]);
        memcpy(o->st[l], keep[l], o->nc[l]);
    }
    double* save[LMAX + 1];
    for (l = lb; l <= L; l++) {
        save[l] = o->Q0[l];
        o->Q0[l] = T[l];
    }
    Ctx x0 = {lb, 0, lb};
    for (l = lb + 1; l <= L; l++)
        for (id = 0; id < o->nc[l]; id++) {
            if (o->st[l][id] != 0) continue;
            coords(o, l, id, c);
            predict_cell(o, l, c, &x0, T[l] + id * m);
            o->st[l][id] = 1; /* filled: usable as a prediction source below */
        }
    for (l = lb; l <= L; l++) {
        o->Q0[l] = save[l];
        free(o->st[l]);
        o->st[l] = keep[l];
    }
    for (id = 0; id < o->nc[L]; id++)
        for (v = 0; v < m; v++) out[(long)v * o->nc[L] + id] = T[L][id * m + v];
    for (l = lb; l <= L; l++) free(T[l]);
}

int or_read(void* h, int what, void* buf, size_t cap, size_t* used)
{
    Orc* o = (Orc*)h;
    int l, v, c[3];
    long id;
    if (!o) return OR_E_INVALID;
    long nleaf = 0;
    for (l = o->lb; l <= o->L; l++)
        for (id = 0; id < o->nc[l]; id++) nleaf += o->st[l][id] == 1;
    size_t need = 0;
    if (what == OR_READ_LEAF_KEYS) need = (size_t)nleaf * 4 * sizeof(int);
    else if (what == OR_READ_LEAF_VALUES) need = (size_t)nleaf * o->m * sizeof(double);
    else if (what == OR_READ_UNIFORM) need = (size_t)o->nc[o->L] * o->m * sizeof(double);
    else if (what == OR_READ_STATS) need = 64 * sizeof(double);
    else if (what == OR_READ_FIELDS) need = (size_t)nleaf * 8 * o->m * sizeof(double);
    else if (what == OR_READ_NODES) {
        long ninner = 0;
        for (l = o->lb; l <= o->L; l++)
            for (id = 0; id < o->nc[l]; id++) ninner += o->st[l][id] == 2;
        need = (size_t)ninner * (4 + 7 * o->m) * sizeof(double);
    } else return OR_E_INVALID;
    if (used) *used = need;
    if (!buf) return OR_OK;
    if (cap < need) return OR_E_INVALID;
    if (what == OR_READ_NODES) { /* per internal node: l i j k, Q0 Q1 Q2 QE XH N1 N3 */
        long i = 0;
        int m = o->m, f;
        for (l = o->lb; l <= o->L; l++)
            for (id = 0; id < o->nc[l]; id++) {
                if (o->st[l][id] != 2) continue;
                double* row = (double*)buf + i * (4 + 7 * m);
                double** F[7] = {o->Q0, o->Q1, o->Q2, o->QE, o->XH, o->N1, o->N3};
                coords(o, l, id, c);
                row[0] = l;
                row[1] = c[0];
                row[2] = c[1];
                row[3] = c[2];
                for (f = 0; f < 7; f++) memcpy(row + 4 + f * m, V(F[f], l, id), sizeof(double) * m);
                i++;
            }
    } else if (what == OR_READ_FIELDS) { /* per leaf: Q0 Q1 Q2 QE NH N1 N3 QX */
        long i = 0;
        int m = o->m, f;
        for (l = o->lb; l <= o->L; l++)
            for (id = 0; id < o->nc[l]; id++) {
                if (o->st[l][id] != 1) continue;
                double** F[8] = {o->Q0, o->Q1, o->Q2, o->QE, o->NH, o->N1, o->N3, o->QX};
                for (f = 0; f < 8; f++)
                    memcpy((double*)buf + (i * 8 + f) * m, V(F[f], l, id), sizeof(double) * m);
                i++;
            }
    } else if (what == OR_READ_LEAF_KEYS || what == OR_READ_LEAF_VALUES) {
        long i = 0;
        for (l = o->lb; l <= o->L; l++)
            for (id = 0; id < o->nc[l]; id++) {
                if (o->st[l][id] != 1) continue;
                if (what == OR_READ_LEAF_KEYS) {
                    int* K = (int*)buf + i * 4;
                    coords(o, l, id, c);
                    K[0] = l;
                    K[1] = c[0];
                    K[2] = c[1];
                    K[3] = c[2];
                } else {
                    memcpy((double*)buf + i * o->m, V(o->QE, l, id), sizeof(double) * o->m);
                }
                i++;
            }
    } else if (what == OR_READ_UNIFORM) {
        uniform(o, (double*)buf);
    } else {
        double* S = (double*)buf;
        memset(S, 0, 64 * sizeof(double));
        S[0] = o->t;
        S[1] = (double)o->iters;
        S[2] = (double)o->macros;
        S[3] = o->dt;
        S[4] = (double)nleaf;
        S[6] = (double)o->near;
        S[7] = (double)o->updates;
        S[15] = (double)o->pos;
        long nodes = 0;
        for (l = o->lb; l <= o->L; l++)
            for (id = 0; id < o->nc[l]; id++) {
                if (o->st[l][id] == 0) continue;
                nodes++;
                if (o->st[l][id] != 1) continue;
                S[16 + l] += 1.0;
                for (v = 0; v < o->m; v++) S[8 + v] += V(o->QE, l, id)[v] * o->vol[l];
            }
        S[5] = (double)nodes;
    }
    return o->bad ? OR_E_STATE : OR_OK;
}

void or_destroy(void* h)
{
    Orc* o = (Orc*)h;
    if (!o) return;
    free_all(o);
    free(o);
}

int or_num_flux(const or_config* cfg, int k, double dxf, const double* W, double* F)
{
    if (!cfg || !W || !F || cfg->dim < 1 || cfg->dim > 3 || k < 0 || k >= cfg->dim || cfg->equation < 0 ||
        cfg->equation > 3 || cfg->flux < 0 || cfg->flux > 1 || (cfg->flux == 1 && cfg->equation != 2))
        return OR_E_INVALID;
    Orc o;
    memset(&o, 0, sizeof o);
    o.cfg = *cfg;
    o.d = cfg->dim;
    o.m = cfg->equation == 2 ? cfg->dim + 2 : 1;
    o.eq = cfg->equation;
    double w[4][MMAX];
    int i, v;
    for (i = 0; i < 4; i++)
        for (v = 0; v < o.m; v++) w[i][v] = W[i * o.m + v];
    num_flux(&o, k, dxf, w, F);
    return OR_OK;
}

const char* or_last_error(void* h)
{
    Orc* o = (Orc*)h;
    return o ? o->err : "null handle";
}
