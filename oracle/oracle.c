/*
 * oracle.c -- plain FP64 CPU oracle for per-point rank-one convexification.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py may load this library.  The CUDA product path shares no code,
 * header, table or constant generator with it.
 *
 * Every function follows the paper (arXiv 2211.14318) step by step, without
 * blocking, fusion or reordering:
 *   - energy:      Sec. 2, Eqs. (2.1)-(2.9), stress Eq. (2.12);
 *   - line:        Sec. 4.1, Eqs. (4.3)-(4.4) restated per point (symmetric
 *                  1-D grid centred at the point, samples with det <= 0 dropped);
 *   - 1-D hull:    Sec. 4.2, Algorithm 1 (Graham scan);
 *   - min over R:  Sec. 4.1, Eq. (4.3);
 *   - recursion:   Sec. 3.1, Eq. (3.3), realised top-down per point
 *                  (lamination tree of Sec. 4.3 / Algorithm 2);
 *   - derivative:  Sec. 5.3, Eq. (5.2) and Algorithm 3.
 *
 * Readings of the paper (where it is silent or garbled) are named at the
 * point of use, each with the reading taken.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off (no FMA contraction,
 * so x86_64 and aarch64 hosts give identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Types (the oracle's own; deliberately not the C-ABI's header).            */
/* ------------------------------------------------------------------------- */

typedef struct {
    double mu;      /* Lame mu                                   */
    double lam;     /* Lame lambda                               */
    double Dinf;    /* asymptotic damage D_inf, Eq. (2.6)         */
    double D0;      /* damage saturation D_0, Eq. (2.6)           */
    int32_t energy; /* 0: NH with damage; 1: double-well test energy */
    int32_t pad;
} orc_material;

typedef struct {
    int32_t n_dir;      /* number of rank-one directions R = a (x) b     */
    int32_t L;          /* samples per line (odd)                         */
    const double *dir;  /* n_dir x 4: (a1, a2, b1, b2)                   */
    double t_half;      /* line covers t in [-t_half, t_half]            */
    int32_t depth;      /* lamination depth K                            */
    int32_t round32;    /* 1: hull decisions on samples rounded to FP32  */
    int32_t newton;     /* 1: refine each split by common-tangent Newton */
    int32_t adaptive;   /* > 0: window doublings allowed per node (below)  */
} orc_scan;

/* One node of the per-point lamination tree in heap layout: node i has
 * children 2i+1 (F-) and 2i+2 (F+). */
typedef struct {
    double F[4];     /* F11 F12 F21 F22                                   */
    double w;        /* W(F) in FP64                                      */
    double h;        /* hull value at t=0 along the chosen direction      */
    double xi;       /* weight of F+ in the split (Algorithm 2)          */
    double weight;   /* product of split weights from the root            */
    double margin;   /* decision margin (see orc_scan_node)               */
    int32_t dir;     /* chosen direction index, -1 if not scanned         */
    int32_t m_minus; /* bridge vertex sample index (0..L-1)               */
    int32_t m_plus;
    int32_t flags;   /* bit0 exists, bit1 scanned, bit2 laminated, bit3 leaf */
    int32_t wexp;    /* the node's line window is t_half 2^wexp               */
    int32_t pad;
} orc_node;

enum { ORC_EXISTS = 1, ORC_SCANNED = 2, ORC_LAMINATED = 4, ORC_LEAF = 8, ORC_NEWTON = 16 };
enum { ORC_OK = 0, ORC_NONPOS_DET = 1 };

/* ------------------------------------------------------------------------- */
/* Energy, Sec. 2                                                            */
/* ------------------------------------------------------------------------- */

/* Eq. (2.3): compressible Neo-Hooke in the invariants I1 = tr C and J. */
double orc_psi0_nh(double I1, double J, double mu, double lam)
{
    double lj = log(J);
    return 0.5 * mu * (I1 - 3.0) - mu * lj + 0.5 * lam * lj * lj;
}

/* Eq. (2.6): D(beta) = D_inf (1 - exp(-beta / D_0)). */
double orc_damage(double beta, double Dinf, double D0)
{
    return Dinf * (1.0 - exp(-beta / D0));
}

/* Antiderivative of Eq. (2.6): Dbar(beta) = D_inf (beta + D_0 exp(-beta/D_0)). */
double orc_damage_antiderivative(double beta, double Dinf, double D0)
{
    return Dinf * (beta + D0 * exp(-beta / D0));
}

/* Eq. (2.9) written term by term, as a function of s = psi0(F):
 *   W = psi(F, D) - psi(F_k, D_k) + beta D - beta_k D_k - Dbar + Dbar_k,
 * with psi = (1 - D) psi0 (Eq. 2.4), beta = max(beta_k, s) (Eq. 2.5) and the
 * reading psi(F_k, D_k) = (1 - D_k) beta_k (the history value is the largest
 * effective energy seen so far). */
double orc_W_of_psi0(double s, double beta_k, double Dinf, double D0)
{
    double beta = s > beta_k ? s : beta_k;
    double D = orc_damage(beta, Dinf, D0);
    double Dk = orc_damage(beta_k, Dinf, D0);
    double psi = (1.0 - D) * s;
    double psik = (1.0 - Dk) * beta_k;
    return psi - psik + beta * D - beta_k * Dk
         - orc_damage_antiderivative(beta, Dinf, D0)
         + orc_damage_antiderivative(beta_k, Dinf, D0);
}

/* Plane strain: C = F^T F of the 3x3 deformation diag-embedded F, so that
 * I1 = |F|_F^2 + 1 and J = det F (Eq. 2.1 with F33 = 1). */
static void nh_invariants(const double F[4], double *I1, double *J)
{
    *I1 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2] + F[3] * F[3] + 1.0;
    *J = F[0] * F[3] - F[1] * F[2];
}

double orc_psi0_stvk(double I1, double I2, double mu, double lam);
void orc_invariants(int32_t d, const double *F, double *I1, double *I2, double *J);

/* psi0(F) of the material (Eq. 2.3, or Eq. 2.2 for energy 2), plane strain. */
double orc_psi0_F(const orc_material *m, const double F[4])
{
    if (m->energy == 2) {
        double I1, I2, J;
        orc_invariants(2, F, &I1, &I2, &J);
        return orc_psi0_stvk(I1, I2, m->mu, m->lam);
    }
    double I1, J;
    nh_invariants(F, &I1, &J);
    return orc_psi0_nh(I1, J, m->mu, m->lam);
}

/* Test energy (not in the paper): separable double well
 *   W = (F11^2 - 1)^2 + F12^2 + F21^2 + (F22 - 1)^2,
 * whose rank-one convex envelope is known in closed form. */
static double dw_energy(const double F[4])
{
    double a = F[0] * F[0] - 1.0, d = F[3] - 1.0;
    return a * a + F[1] * F[1] + F[2] * F[2] + d * d;
}

static void stvk_dpsi0(const orc_material *m, int32_t d, const double *F, double *G);

/* Incremental stress potential W(F), Eq. (2.9); NaN where det F <= 0.
 * energy 0: Eq. (2.3); 2: Eq. (2.2) (plane strain); 1: the double well. */
double orc_energy(const orc_material *m, const double F[4], double beta_k)
{
    if (m->energy == 1)
        return dw_energy(F);
    if (m->energy == 2) {
        double I1, I2, J;
        orc_invariants(2, F, &I1, &I2, &J);
        if (!(J > 0.0))
            return NAN;
        return orc_W_of_psi0(orc_psi0_stvk(I1, I2, m->mu, m->lam), beta_k, m->Dinf, m->D0);
    }
    double I1, J;
    nh_invariants(F, &I1, &J);
    if (!(J > 0.0))
        return NAN;
    double s = orc_psi0_nh(I1, J, m->mu, m->lam);
    return orc_W_of_psi0(s, beta_k, m->Dinf, m->D0);
}

/* P = dW/dF, Eq. (2.12).  By the chain rule through s = psi0(F) (beta is the
 * minimiser of Eq. (2.8), so its own variation drops out):
 *   dW/ds = 1 - D(max(s, beta_k)),
 *   dpsi0/dF = mu F - mu F^{-T} + lam ln J F^{-T}. */
void orc_stress(const orc_material *m, const double F[4], double beta_k, double P[4])
{
    if (m->energy == 1) {
        P[0] = 4.0 * F[0] * (F[0] * F[0] - 1.0);
        P[1] = 2.0 * F[1];
        P[2] = 2.0 * F[2];
        P[3] = 2.0 * (F[3] - 1.0);
        return;
    }
    if (m->energy == 2) {
        double I1, I2, J, G[4];
        orc_invariants(2, F, &I1, &I2, &J);
        if (!(J > 0.0)) {
            P[0] = P[1] = P[2] = P[3] = NAN;
            return;
        }
        double s = orc_psi0_stvk(I1, I2, m->mu, m->lam);
        double beta = s > beta_k ? s : beta_k;
        double g = 1.0 - orc_damage(beta, m->Dinf, m->D0);
        stvk_dpsi0(m, 2, F, G);
        for (int i = 0; i < 4; ++i)
            P[i] = g * G[i];
        return;
    }
    double I1, J;
    nh_invariants(F, &I1, &J);
    if (!(J > 0.0)) {
        P[0] = P[1] = P[2] = P[3] = NAN;
        return;
    }
    double s = orc_psi0_nh(I1, J, m->mu, m->lam);
    double beta = s > beta_k ? s : beta_k;
    double g = 1.0 - orc_damage(beta, m->Dinf, m->D0);
    /* F^{-T} = cof F / J, with cof F = [[F22, -F21], [-F12, F11]] */
    double FiT[4] = {F[3] / J, -F[2] / J, -F[1] / J, F[0] / J};
    double lj = log(J);
    for (int i = 0; i < 4; ++i)
        P[i] = g * (m->mu * F[i] - m->mu * FiT[i] + m->lam * lj * FiT[i]);
}

/* Tangent A = d^2 W / dF dF (4 x 4, A[4 i + k] = d P_i / d F_k, F flattened
 * row-major).  Differentiating P = g(s) dpsi0/dF with g = 1 - D(max(s, beta_k)):
 *   A = g d^2 psi0/dF^2 + [s > beta_k] g'(s) dpsi0/dF (x) dpsi0/dF,
 * g'(s) = -D'(s) = -(D_inf / D_0) exp(-s / D_0), and for Eq. (2.3)
 *   d^2 psi0 / dF_iJ dF_kL = mu d_ik d_JL + (mu - lam ln J) Fit_iL Fit_kJ
 *                           + lam Fit_iJ Fit_kL,     Fit = F^{-T},
 * from d(F^{-T})_iJ / dF_kL = -Fit_iL Fit_kJ and d ln J / dF = F^{-T}. */
void orc_tangent(const orc_material *m, const double F[4], double beta_k, double A[16])
{
    if (m->energy == 2) { /* not built for Eq. (2.2) */
        for (int i = 0; i < 16; ++i)
            A[i] = NAN;
        return;
    }
    if (m->energy == 1) {
        for (int i = 0; i < 16; ++i)
            A[i] = 0.0;
        A[0] = 12.0 * F[0] * F[0] - 4.0;
        A[5] = 2.0;
        A[10] = 2.0;
        A[15] = 2.0;
        return;
    }
    double I1, J;
    nh_invariants(F, &I1, &J);
    if (!(J > 0.0)) {
        for (int i = 0; i < 16; ++i)
            A[i] = NAN;
        return;
    }
    double s = orc_psi0_nh(I1, J, m->mu, m->lam);
    double beta = s > beta_k ? s : beta_k;
    double g = 1.0 - orc_damage(beta, m->Dinf, m->D0);
    double lj = log(J);
    double Fit[2][2] = {{F[3] / J, -F[2] / J}, {-F[1] / J, F[0] / J}};
    double dpsi[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            dpsi[2 * i + j] = m->mu * F[2 * i + j] - m->mu * Fit[i][j] + m->lam * lj * Fit[i][j];
    double gp = s > beta_k ? -(m->Dinf / m->D0) * exp(-s / m->D0) : 0.0;
    for (int i = 0; i < 2; ++i)
        for (int J1 = 0; J1 < 2; ++J1)
            for (int k = 0; k < 2; ++k)
                for (int L1 = 0; L1 < 2; ++L1) {
                    double d2 = (i == k && J1 == L1 ? m->mu : 0.0)
                              + (m->mu - m->lam * lj) * Fit[i][L1] * Fit[k][J1]
                              + m->lam * Fit[i][J1] * Fit[k][L1];
                    A[4 * (2 * i + J1) + (2 * k + L1)] =
                        g * d2 + gp * dpsi[2 * i + J1] * dpsi[2 * k + L1];
                }
}

/* History update between load steps, Eq. (2.5): beta_new = max(beta_k, psi0(F)). */
void orc_history_update(const orc_material *m, int64_t n, const double *F,
                        const double *beta_in, double *beta_out)
{
    for (int64_t p = 0; p < n; ++p) {
        double s = orc_psi0_F(m, F + 4 * p);
        double b = beta_in ? beta_in[p] : 0.0;
        beta_out[p] = s > b ? s : b;
    }
}

/* ------------------------------------------------------------------------- */
/* Rank-one lines, Sec. 4.1, Eq. (4.4) restated per point                    */
/* ------------------------------------------------------------------------- */

/* Direction table for the angle grid: a_i = (cos(pi i/Na), sin(pi i/Na)),
 * b_j likewise, direction index j_dir = i * Nb + j. */
void orc_angle_directions(int32_t Na, int32_t Nb, double *dir)
{
    for (int i = 0; i < Na; ++i) {
        double ta = M_PI * (double)i / (double)Na;
        for (int j = 0; j < Nb; ++j) {
            double tb = M_PI * (double)j / (double)Nb;
            double *d = dir + 4 * ((int64_t)i * Nb + j);
            d[0] = cos(ta);
            d[1] = sin(ta);
            d[2] = cos(tb);
            d[3] = sin(tb);
        }
    }
}

/* R = a (x) b, row-major (R11 R12 R21 R22). */
static void rank_one(const double *d, double R[4])
{
    R[0] = d[0] * d[2];
    R[1] = d[0] * d[3];
    R[2] = d[1] * d[2];
    R[3] = d[1] * d[3];
}

/* Samples of W along F + t_m R, t_m = (m - m0) h, h = 2 t_half / (L - 1),
 * m0 = (L - 1) / 2.  valid[m] = 0 where det(F + t_m R) <= 0 (NH only). */
void orc_sample_line(const orc_material *mat, const double F[4], double beta_k,
                     const double R[4], int32_t L, double t_half, int32_t round32,
                     double *w, uint8_t *valid)
{
    int m0 = (L - 1) / 2;
    double h = 2.0 * t_half / (double)(L - 1);
    for (int m = 0; m < L; ++m) {
        double t = (double)(m - m0) * h;
        double G[4];
        for (int i = 0; i < 4; ++i)
            G[i] = F[i] + t * R[i];
        double v = orc_energy(mat, G, beta_k);
        if (mat->energy != 1 && !(G[0] * G[3] - G[1] * G[2] > 0.0)) {
            valid[m] = 0;
            w[m] = NAN;
            continue;
        }
        valid[m] = 1;
        w[m] = round32 ? (double)(float)v : v;
    }
}

/* ------------------------------------------------------------------------- */
/* One-dimensional convexification, Sec. 4.2, Algorithm 1                    */
/* ------------------------------------------------------------------------- */

/* Algorithm 1 (Graham scan) on points (x[i], w[i]), x strictly increasing.
 * Writes the indices of the hull vertices to vtx and returns their number.
 * Readings: the start uses the first two points (x, w); the pop loop runs
 * while at least two vertices remain; ">=" pops collinear points, so the
 * returned vertices are strict. */
int32_t orc_lower_hull(int32_t n, const double *x, const double *w, int32_t *vtx)
{
    if (n <= 0)
        return 0;
    vtx[0] = 0;
    if (n == 1)
        return 1;
    vtx[1] = 1;
    int32_t k = 2;
    for (int32_t i = 2; i < n; ++i) {
        while (k >= 2) {
            int32_t p = vtx[k - 2], q = vtx[k - 1];
            /* slope(p->q) >= slope(q->i)  <=>  q is not strictly below */
            if ((w[q] - w[p]) * (x[i] - x[q]) >= (w[i] - w[q]) * (x[q] - x[p]))
                --k;
            else
                break;
        }
        vtx[k++] = i;
    }
    return k;
}

/* Hull of the valid samples of one line, read at x = 0 (the point F itself).
 * Abscissae are the integers m - m0.  Returns the value at 0 and the bridge
 * vertices m_minus <= m0 <= m_plus (both m0 when m0 is itself a vertex).
 * If margin_out is non-NULL it receives the decision margin: the largest eps
 * such that perturbing every sample by at most eps cannot change the result
 *  - bridge a < 0 < b:  min over other samples i of
 *        (w_i - chord(x_i)) / (1 + (|x_i - x_a| + |x_i - x_b|) / (x_b - x_a));
 *  - vertex at 0:       (hull of the samples without m0, read at 0, - w_m0) / 2
 *                       (+inf when one side is empty). */
double orc_line_bridge(int32_t L, const double *w, const uint8_t *valid,
                       int32_t *m_minus, int32_t *m_plus, double *margin_out)
{
    int32_t m0 = (L - 1) / 2;
    double *xs = (double *)malloc(sizeof(double) * L);
    double *ws = (double *)malloc(sizeof(double) * L);
    int32_t *id = (int32_t *)malloc(sizeof(int32_t) * L);
    int32_t *vtx = (int32_t *)malloc(sizeof(int32_t) * L);
    int32_t n = 0;
    for (int32_t m = 0; m < L; ++m)
        if (valid[m]) {
            xs[n] = (double)(m - m0);
            ws[n] = w[m];
            id[n] = m;
            ++n;
        }
    int32_t nv = orc_lower_hull(n, xs, ws, vtx);
    double h = w[m0];
    int32_t a = m0, b = m0;
    for (int32_t k = 0; k + 1 < nv; ++k) {
        double xa = xs[vtx[k]], xb = xs[vtx[k + 1]];
        if (xa < 0.0 && xb > 0.0) {
            a = id[vtx[k]];
            b = id[vtx[k + 1]];
            /* linear interpolation of the hull at x = 0 */
            h = (xb * ws[vtx[k]] - xa * ws[vtx[k + 1]]) / (xb - xa);
            break;
        }
    }
    *m_minus = a;
    *m_plus = b;
    if (margin_out) {
        double mg = INFINITY;
        if (a != b) {
            double xa = (double)(a - m0), xb = (double)(b - m0);
            for (int32_t i = 0; i < n; ++i) {
                if (id[i] == a || id[i] == b)
                    continue;
                double x = xs[i];
                double chord = (w[a] * (xb - x) + w[b] * (x - xa)) / (xb - xa);
                double kappa = (fabs(x - xa) + fabs(x - xb)) / (xb - xa);
                double r = (ws[i] - chord) / (1.0 + kappa);
                if (r < mg)
                    mg = r;
            }
        } else {
            /* hull of all valid samples except m0, read at 0 */
            int32_t n2 = 0;
            for (int32_t i = 0; i < n; ++i)
                if (id[i] != m0) {
                    xs[n2] = xs[i];
                    ws[n2] = ws[i];
                    ++n2;
                }
            int32_t nv2 = orc_lower_hull(n2, xs, ws, vtx);
            double h2 = INFINITY;
            for (int32_t k = 0; k + 1 < nv2; ++k) {
                double xa = xs[vtx[k]], xb = xs[vtx[k + 1]];
                if (xa < 0.0 && xb > 0.0) {
                    h2 = (xb * ws[vtx[k]] - xa * ws[vtx[k + 1]]) / (xb - xa);
                    break;
                }
            }
            mg = 0.5 * (h2 - w[m0]);
        }
        *margin_out = mg;
    }
    free(xs);
    free(ws);
    free(id);
    free(vtx);
    return h;
}

/* ------------------------------------------------------------------------- */
/* Minimum over directions, Sec. 4.1, Eq. (4.3)                              */
/* ------------------------------------------------------------------------- */

/* Scans every direction at one node F.  For direction j: h_j, bridge
 * (m_minus_j, m_plus_j).  The node picks j* = argmin h_j (lowest j on equal
 * values) and laminates iff the bridge at j* excludes m0.
 * Optional per-direction outputs (NULL to skip).
 * The node margin is min(bridge margin at j*, (h_(2) - h_(1)) / 2) for a
 * laminating node and min_j (no-lamination margin of j) otherwise. */
int32_t orc_scan_node(const orc_material *mat, const orc_scan *sc, const double F[4],
                      double beta_k, double *h_out, int32_t *mm_out, int32_t *mp_out,
                      double *margin_dir_out, double *h_best, int32_t *m_minus,
                      int32_t *m_plus, double *node_margin)
{
    int32_t L = sc->L;
    if (sc->n_dir <= 0)
        return -1;
    double *w = (double *)malloc(sizeof(double) * L);
    uint8_t *valid = (uint8_t *)malloc(L);
    double *hs = (double *)malloc(sizeof(double) * sc->n_dir);
    double *mg = (double *)malloc(sizeof(double) * sc->n_dir);
    int32_t *mm = (int32_t *)malloc(sizeof(int32_t) * sc->n_dir);
    int32_t *mp = (int32_t *)malloc(sizeof(int32_t) * sc->n_dir);
    for (int32_t j = 0; j < sc->n_dir; ++j) {
        double R[4];
        rank_one(sc->dir + 4 * j, R);
        orc_sample_line(mat, F, beta_k, R, L, sc->t_half, sc->round32, w, valid);
        hs[j] = orc_line_bridge(L, w, valid, &mm[j], &mp[j], &mg[j]);
    }
    int32_t best = 0;
    for (int32_t j = 1; j < sc->n_dir; ++j)
        if (hs[j] < hs[best])
            best = j;
    int32_t m0 = (L - 1) / 2;
    int laminated = mm[best] != m0;
    double margin;
    if (laminated) {
        double second = INFINITY;
        for (int32_t j = 0; j < sc->n_dir; ++j)
            if (j != best && hs[j] < second)
                second = hs[j];
        margin = mg[best];
        double g = 0.5 * (second - hs[best]);
        if (g < margin)
            margin = g;
    } else {
        margin = INFINITY;
        for (int32_t j = 0; j < sc->n_dir; ++j)
            if (mg[j] < margin)
                margin = mg[j];
    }
    if (h_out)
        memcpy(h_out, hs, sizeof(double) * sc->n_dir);
    if (mm_out)
        memcpy(mm_out, mm, sizeof(int32_t) * sc->n_dir);
    if (mp_out)
        memcpy(mp_out, mp, sizeof(int32_t) * sc->n_dir);
    if (margin_dir_out)
        memcpy(margin_dir_out, mg, sizeof(double) * sc->n_dir);
    *h_best = hs[best];
    *m_minus = mm[best];
    *m_plus = mp[best];
    *node_margin = margin;
    free(w);
    free(valid);
    free(hs);
    free(mg);
    free(mm);
    free(mp);
    return best;
}

/* ------------------------------------------------------------------------- */
/* Optional refinement of a split: common tangent by Newton (a reading: the  */
/* paper solves for laminates on grids only)                                 */
/* ------------------------------------------------------------------------- */

/* g(t) = W(F + t R) and its first two derivatives g' = P : R, g'' = R : A : R. */
static void line_derivs(const orc_material *m, const double F[4], double beta_k,
                        const double R[4], double t, double *g, double *g1, double *g2)
{
    double G[4], P[4], A[16];
    for (int i = 0; i < 4; ++i)
        G[i] = F[i] + t * R[i];
    *g = orc_energy(m, G, beta_k);
    orc_stress(m, G, beta_k, P);
    orc_tangent(m, G, beta_k, A);
    *g1 = 0.0;
    *g2 = 0.0;
    for (int i = 0; i < 4; ++i) {
        *g1 += P[i] * R[i];
        for (int k = 0; k < 4; ++k)
            *g2 += R[i] * A[4 * i + k] * R[k];
    }
}

/* Chord value at t = 0 of the segment from (t-, g(t-)) to (t+, g(t+)). */
static double chord_at_zero(double tm, double gm, double tp, double gp)
{
    return gm + (gp - gm) * (0.0 - tm) / (tp - tm);
}

/* Newton on the common-tangent conditions of the split (t-, t+) along R:
 *   f1 = g'(t-) - g'(t+) = 0,
 *   f2 = g'(t-) (t+ - t-) - (g(t+) - g(t-)) = 0,
 * i.e. one line touches g at both ends (the stationarity conditions of the
 * chord value at 0 over continuous t-, t+).  Seeded by the grid bridge, at
 * most 8 iterations.  Accepted (returns 1) only if it converged with
 * -t_half <= t- < 0 < t+ <= t_half, det F > 0 at both ends and a chord value
 * at 0 not above the grid's; otherwise returns 0 and leaves the outputs. */
int32_t orc_newton_tangent(const orc_material *m, const double F[4], double beta_k,
                           const double R[4], double t_half, double tm0, double tp0,
                           double h_grid, double *tm_out, double *tp_out, double *h_out)
{
    if (m->energy == 2) /* line derivatives are written for Eq. (2.3) only */
        return 0;
    double tm = tm0, tp = tp0;
    int converged = 0;
    for (int it = 0; it < 8; ++it) {
        double gm, gm1, gm2, gp, gp1, gp2;
        line_derivs(m, F, beta_k, R, tm, &gm, &gm1, &gm2);
        line_derivs(m, F, beta_k, R, tp, &gp, &gp1, &gp2);
        double f1 = gm1 - gp1;
        double f2 = gm1 * (tp - tm) - (gp - gm);
        /* Jacobian d(f1, f2) / d(t-, t+) */
        double j11 = gm2, j12 = -gp2;
        double j21 = gm2 * (tp - tm), j22 = gm1 - gp1;
        double det = j11 * j22 - j12 * j21;
        if (!(fabs(det) > 0.0) || !isfinite(det))
            return 0;
        double dm = (-f1 * j22 + f2 * j12) / det;
        double dp = (-f2 * j11 + f1 * j21) / det;
        tm += dm;
        tp += dp;
        if (!isfinite(tm) || !isfinite(tp))
            return 0;
        if (fabs(dm) <= 1e-13 * (1.0 + fabs(tm)) && fabs(dp) <= 1e-13 * (1.0 + fabs(tp))) {
            converged = 1;
            break;
        }
    }
    if (!converged)
        return 0;
    if (!(tm >= -t_half && tm < 0.0 && tp > 0.0 && tp <= t_half))
        return 0;
    double gm = 0.0, gp = 0.0, d1, d2;
    line_derivs(m, F, beta_k, R, tm, &gm, &d1, &d2);
    line_derivs(m, F, beta_k, R, tp, &gp, &d1, &d2);
    if (!isfinite(gm) || !isfinite(gp))
        return 0;
    double h = chord_at_zero(tm, gm, tp, gp);
    if (!(h <= h_grid))
        return 0;
    *tm_out = tm;
    *tp_out = tp;
    *h_out = h;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Lamination to depth K, Eq. (3.3), and derivative, Eq. (5.2)/Algorithm 3   */
/* ------------------------------------------------------------------------- */

/* Node value V_K(G) (reading of "lamination depth" for a per-point method):
 *   V_0(G) = W(G);
 *   V_K(G) = W(G)                              if G does not laminate;
 *   V_K(G) = xi V_{K-1}(F+) + (1-xi) V_{K-1}(F-) otherwise,
 * with (R*, F+-, xi) from the line scan of W at G.  The tree is stored in
 * heap layout; leaves carry the product of split weights (Algorithm 2's xi).
 *
 * Adaptive window (sc->adaptive > 0; Sec. 4.1 asks for a radius r
 * "sufficiently large"): a node whose split has an end on the end of its line
 * is scanned again with the line window doubled (t_half 2^e, the same L), at
 * most sc->adaptive doublings; the node's children start from its window. */
static void build_tree(const orc_material *mat, const orc_scan *sc, double beta_k,
                       orc_node *tree, int32_t i, int32_t depth_left, int32_t e0)
{
    orc_node *nd = &tree[i];
    nd->w = orc_energy(mat, nd->F, beta_k);
    nd->flags |= ORC_EXISTS;
    nd->dir = -1;
    nd->m_minus = nd->m_plus = (sc->L - 1) / 2;
    nd->h = nd->w;
    nd->xi = 0.0;
    nd->margin = INFINITY;
    nd->wexp = e0;
    if (depth_left == 0) {
        nd->flags |= ORC_LEAF;
        return;
    }
    double h, margin;
    int32_t mm, mp, j;
    int32_t m0 = (sc->L - 1) / 2;
    int32_t e = e0;
    orc_scan sce = *sc;
    for (;;) {
        sce.t_half = ldexp(sc->t_half, e);
        j = orc_scan_node(mat, &sce, nd->F, beta_k, NULL, NULL, NULL, NULL, &h, &mm, &mp, &margin);
        if (mm != m0 && (mm == 0 || mp == sc->L - 1) && e < sc->adaptive) {
            ++e;
            continue;
        }
        break;
    }
    nd->wexp = e;
    nd->flags |= ORC_SCANNED;
    nd->dir = j;
    nd->h = h;
    nd->m_minus = mm;
    nd->m_plus = mp;
    nd->margin = margin;
    if (mm == m0) {
        nd->flags |= ORC_LEAF;
        return;
    }
    nd->flags |= ORC_LAMINATED;
    double R[4];
    rank_one(sc->dir + 4 * j, R);
    double hstep = 2.0 * sce.t_half / (double)(sc->L - 1);
    double tm = (double)(mm - m0) * hstep, tp = (double)(mp - m0) * hstep;
    /* Algorithm 2: xi = |F - F-|_1 / |F+ - F-|_1 = (m0 - m-)/(m+ - m-) */
    nd->xi = (double)(m0 - mm) / (double)(mp - mm);
    double tmN, tpN, hN;
    if (sc->newton &&
        orc_newton_tangent(mat, nd->F, beta_k, R, sce.t_half, tm, tp, h, &tmN, &tpN, &hN)) {
        tm = tmN;
        tp = tpN;
        nd->h = hN;
        nd->xi = (0.0 - tm) / (tp - tm);
        nd->flags |= ORC_NEWTON;
    }
    orc_node *cm = &tree[2 * i + 1], *cp = &tree[2 * i + 2];
    for (int k = 0; k < 4; ++k) {
        cm->F[k] = nd->F[k] + tm * R[k];
        cp->F[k] = nd->F[k] + tp * R[k];
    }
    cm->weight = nd->weight * (1.0 - nd->xi);
    cp->weight = nd->weight * nd->xi;
    build_tree(mat, sc, beta_k, tree, 2 * i + 1, depth_left - 1, e);
    build_tree(mat, sc, beta_k, tree, 2 * i + 2, depth_left - 1, e);
}

/* Algorithm 3: recursive evaluation of W, P as the xi-weighted sum over
 * children; leaves evaluate the non-convex W and its derivative. */
static void eval_tree(const orc_material *mat, double beta_k, const orc_node *tree,
                      int32_t i, double *W, double P[4])
{
    const orc_node *nd = &tree[i];
    if (!(nd->flags & ORC_LAMINATED)) {
        *W = orc_energy(mat, nd->F, beta_k);
        orc_stress(mat, nd->F, beta_k, P);
        return;
    }
    double Wm, Wp, Pm[4], Pp[4];
    eval_tree(mat, beta_k, tree, 2 * i + 1, &Wm, Pm);
    eval_tree(mat, beta_k, tree, 2 * i + 2, &Wp, Pp);
    *W = (1.0 - nd->xi) * Wm + nd->xi * Wp;
    for (int k = 0; k < 4; ++k)
        P[k] = (1.0 - nd->xi) * Pm[k] + nd->xi * Pp[k];
}

/* Algorithm 3 for the tangent: the same xi-weighted recursion as eval_tree
 * applied to the second derivative (Eq. 5.2 differentiated once more with
 * the laminate held fixed), leaves evaluating orc_tangent. */
static void eval_tree_tangent(const orc_material *mat, double beta_k, const orc_node *tree,
                              int32_t i, double A[16])
{
    const orc_node *nd = &tree[i];
    if (!(nd->flags & ORC_LAMINATED)) {
        orc_tangent(mat, nd->F, beta_k, A);
        return;
    }
    double Am[16], Ap[16];
    eval_tree_tangent(mat, beta_k, tree, 2 * i + 1, Am);
    eval_tree_tangent(mat, beta_k, tree, 2 * i + 2, Ap);
    for (int k = 0; k < 16; ++k)
        A[k] = (1.0 - nd->xi) * Am[k] + nd->xi * Ap[k];
}

/* Tangent of W^R at n points from their trees (n x (2^{K+1}-1) nodes, the
 * layout orc_convexify writes; the tree's xi fields are used). */
void orc_tree_tangent(const orc_material *mat, int32_t depth, int64_t n, const orc_node *tree,
                      const double *beta_k, double *A)
{
    int32_t nt = (1 << (depth + 1)) - 1;
    for (int64_t p = 0; p < n; ++p) {
        if (!(tree[p * nt].flags & ORC_EXISTS)) {
            for (int k = 0; k < 16; ++k)
                A[16 * p + k] = NAN;
            continue;
        }
        eval_tree_tangent(mat, beta_k[p], tree + p * nt, 0, A + 16 * p);
    }
}

int32_t orc_tree_size(int32_t depth)
{
    return (1 << (depth + 1)) - 1;
}

/* Per-point convexification: W^R, P and the tree (n x (2^{K+1}-1) nodes,
 * may be NULL).  status[p] = 1 where det F <= 0 (W^R, P = NaN). */
void orc_convexify(const orc_material *mat, const orc_scan *sc, int64_t n, const double *F,
                   const double *beta_k, double *W_R, double *P, orc_node *tree,
                   int32_t *status, int32_t nthreads)
{
    int32_t nt = orc_tree_size(sc->depth);
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t p = 0; p < n; ++p) {
        orc_node *tr = tree ? tree + p * nt : (orc_node *)calloc(nt, sizeof(orc_node));
        if (tree)
            memset(tr, 0, sizeof(orc_node) * nt);
        const double *Fp = F + 4 * p;
        double J = Fp[0] * Fp[3] - Fp[1] * Fp[2];
        if (mat->energy != 1 && !(J > 0.0)) {
            W_R[p] = NAN;
            for (int k = 0; k < 4; ++k)
                P[4 * p + k] = NAN;
            status[p] = ORC_NONPOS_DET;
            if (!tree)
                free(tr);
            continue;
        }
        memcpy(tr[0].F, Fp, sizeof(double) * 4);
        tr[0].weight = 1.0;
        build_tree(mat, sc, beta_k[p], tr, 0, sc->depth, 0);
        eval_tree(mat, beta_k[p], tr, 0, &W_R[p], P + 4 * p);
        status[p] = ORC_OK;
        if (!tree)
            free(tr);
    }
}

int32_t orc_node_size(void)
{
    return (int32_t)sizeof(orc_node);
}

/* ------------------------------------------------------------------------- */
/* St. Venant-Kirchhoff (Eq. 2.2) and the three-dimensional invariants        */
/* ------------------------------------------------------------------------- */

/* Eq. (2.2): psi0 = lam/8 (I1 - 3)^2 + mu/4 (I1^2 - 2 I1 - 2 I2 + 3). */
double orc_psi0_stvk(double I1, double I2, double mu, double lam)
{
    return lam / 8.0 * (I1 - 3.0) * (I1 - 3.0) + mu / 4.0 * (I1 * I1 - 2.0 * I1 - 2.0 * I2 + 3.0);
}

/* C = F^T F of F in R^{d x d} (row-major), d = 2 or 3. */
static void right_cauchy_green(int32_t d, const double *F, double *C)
{
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double c = 0.0;
            for (int k = 0; k < d; ++k)
                c += F[d * k + i] * F[d * k + j];
            C[d * i + j] = c;
        }
}

static double det3(const double *F)
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6])
         + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* Cofactor matrix of a 3 x 3 F (d det F / dF); F^{-T} = cof F / det F. */
static void cof3(const double *F, double *c)
{
    c[0] = F[4] * F[8] - F[5] * F[7];
    c[1] = F[5] * F[6] - F[3] * F[8];
    c[2] = F[3] * F[7] - F[4] * F[6];
    c[3] = F[2] * F[7] - F[1] * F[8];
    c[4] = F[0] * F[8] - F[2] * F[6];
    c[5] = F[1] * F[6] - F[0] * F[7];
    c[6] = F[1] * F[5] - F[2] * F[4];
    c[7] = F[2] * F[3] - F[0] * F[5];
    c[8] = F[0] * F[4] - F[1] * F[3];
}

/* Invariants of Sec. 2 for F in R^{d x d}: I1 = tr C, I2 = tr Cof C (the sum of
 * the principal 2 x 2 minors of C), J = det F.  d = 2 is plane strain: C is
 * embedded with C33 = 1, so I1 gains 1 and I2 gains C11 + C22. */
void orc_invariants(int32_t d, const double *F, double *I1, double *I2, double *J)
{
    double C[9];
    right_cauchy_green(d, F, C);
    if (d == 2) {
        *I1 = C[0] + C[3] + 1.0;
        *I2 = (C[0] * C[3] - C[1] * C[2]) + C[0] + C[3];
        *J = F[0] * F[3] - F[1] * F[2];
    } else {
        *I1 = C[0] + C[4] + C[8];
        *I2 = (C[0] * C[4] - C[1] * C[3]) + (C[0] * C[8] - C[2] * C[6])
            + (C[4] * C[8] - C[5] * C[7]);
        *J = det3(F);
    }
}

/* psi0 of the material at F in R^{d x d}: Eq. (2.3) (energy 0) with |J|
 * (the caller decides what det F <= 0 means), or Eq. (2.2) (energy 2). */
static double psi0_d(const orc_material *m, int32_t d, const double *F, double *Jout)
{
    double I1, I2, J;
    if (d == 2 && m->energy == 0) {
        nh_invariants(F, &I1, &J);
        *Jout = J;
        return orc_psi0_nh(I1, fabs(J), m->mu, m->lam);
    }
    orc_invariants(d, F, &I1, &I2, &J);
    *Jout = J;
    if (m->energy == 2)
        return orc_psi0_stvk(I1, I2, m->mu, m->lam);
    return orc_psi0_nh(I1, fabs(J), m->mu, m->lam);
}

/* dpsi0/dF at F in R^{d x d} (d x d entries):
 *   Eq. (2.3): mu F - mu F^{-T} + lam ln|J| F^{-T}  (d ln|J| / dF = F^{-T});
 *   Eq. (2.2): F (lam/2 (I1 - 3) 1 + mu (C - 1)) (2 F dpsi0/dC with
 *              dI1/dC = 1, dI2/dC = I1 1 - C; the d x d blocks of C and 1). */
static void stvk_dpsi0(const orc_material *m, int32_t d, const double *F, double *G)
{
    double I1, I2, J;
    orc_invariants(d, F, &I1, &I2, &J);
    {
        double C[9], S[9];
        right_cauchy_green(d, F, C);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                S[d * i + j] = m->mu * (C[d * i + j] - (i == j ? 1.0 : 0.0))
                             + (i == j ? 0.5 * m->lam * (I1 - 3.0) : 0.0);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double g = 0.0;
                for (int k = 0; k < d; ++k)
                    g += F[d * i + k] * S[d * k + j];
                G[d * i + j] = g;
            }
    }
}

static void dpsi0_d(const orc_material *m, int32_t d, const double *F, double *G)
{
    int D = d * d;
    if (m->energy == 2) {
        stvk_dpsi0(m, d, F, G);
        return;
    }
    double I1, I2, J;
    orc_invariants(d, F, &I1, &I2, &J);
    double c[9];
    if (d == 2) {
        c[0] = F[3];
        c[1] = -F[2];
        c[2] = -F[1];
        c[3] = F[0];
    } else {
        cof3(F, c);
    }
    double lj = log(fabs(J));
    for (int k = 0; k < D; ++k) {
        double fit = c[k] / J;
        G[k] = m->mu * F[k] - m->mu * fit + m->lam * lj * fit;
    }
}

/* ------------------------------------------------------------------------- */
/* Global-grid rank-one convexification: Eq. (4.3) on the cuboid grid of     */
/* Sec. 5.2 with the reduced direction set R^1_1 of Eq. (5.1)                */
/* ------------------------------------------------------------------------- */

/* Grid of Sec. 5.2 for F in R^{d x d}: component c of F (row-major, D = d^2
 * components) takes the values lo[c] + i delta[c], i = 0 .. n[c] - 1; flat
 * index with the last component fastest. */
typedef struct {
    int32_t dim;
    int32_t n[9];
    double lo[9];
    double delta[9];
} orc_grid;

static int grid_D(const orc_grid *g)
{
    return g->dim * g->dim;
}

int64_t orc_grid_count(const orc_grid *g)
{
    int64_t N = 1;
    for (int c = 0; c < grid_D(g); ++c)
        N *= g->n[c];
    return N;
}

static void grid_index(const orc_grid *g, int64_t idx, int32_t *i)
{
    for (int c = grid_D(g) - 1; c >= 0; --c) {
        i[c] = (int32_t)(idx % g->n[c]);
        idx /= g->n[c];
    }
}

static int64_t grid_flat(const orc_grid *g, const int32_t *i)
{
    int64_t f = 0;
    for (int c = 0; c < grid_D(g); ++c)
        f = f * g->n[c] + i[c];
    return f;
}

void orc_grid_point(const orc_grid *g, int64_t idx, double *F)
{
    int32_t i[9];
    grid_index(g, idx, i);
    for (int c = 0; c < grid_D(g); ++c)
        F[c] = g->lo[c] + (double)i[c] * g->delta[c];
}

/* Eq. (5.1): a (x) b with a, b in Z^d, |a|_inf = |b|_inf = 1, one of each pair
 * +-a (x) b (the sign of a direction gives the same line), written as the
 * grid-index offset (a_i b_j, row-major) of one step.
 * d = 2: a and b run over (1,0), (0,1), (1,1), (1,-1); direction 4 ia + ib.
 * d = 3 (the reading for the nine-dimensional study of Sec. 6.8): the 13
 * vectors of {-1,0,1}^3 with first nonzero entry +1, in the order axes,
 * face diagonals, body diagonals: (1,0,0), (0,1,0), (0,0,1), (1,1,0), (1,-1,0),
 * (1,0,1), (1,0,-1), (0,1,1), (0,1,-1), (1,1,1), (1,1,-1), (1,-1,1),
 * (1,-1,-1); direction 13 ia + ib, 169 in all. */
void orc_r11_directions(int32_t *off)
{
    static const int32_t v[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
    for (int ia = 0; ia < 4; ++ia)
        for (int ib = 0; ib < 4; ++ib) {
            int32_t *o = off + 4 * (4 * ia + ib);
            o[0] = v[ia][0] * v[ib][0];
            o[1] = v[ia][0] * v[ib][1];
            o[2] = v[ia][1] * v[ib][0];
            o[3] = v[ia][1] * v[ib][1];
        }
}

void orc_r11_directions3(int32_t *off)
{
    static const int32_t v[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                     {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                     {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
    for (int ia = 0; ia < 13; ++ia)
        for (int ib = 0; ib < 13; ++ib) {
            int32_t *o = off + 9 * (13 * ia + ib);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    o[3 * i + j] = v[ia][i] * v[ib][j];
        }
}

/* What det F <= 0 means on the grid (rule), the readings of the studies of
 * Sec. 6.1:
 *   0: excluded (NaN), as on the per-point path;
 *   1: Eq. (2.3) takes ln|det F|, so det F < 0 mirrors det F > 0 (the NH
 *      study); Eq. (2.2) is a polynomial in F and is kept everywhere (the
 *      STVK study); only det F = 0 stays excluded for Eq. (2.3). */

/* Energy at a grid point (d = g->dim); the double well exists for d = 2. */
static double grid_W(const orc_material *m, int32_t d, const double *F, double beta_k,
                     int32_t rule)
{
    if (m->energy == 1)
        return d == 2 ? orc_energy(m, F, beta_k) : NAN;
    if (d == 2 && m->energy == 0 && rule == 0)
        return orc_energy(m, F, beta_k);
    double J;
    double s = psi0_d(m, d, F, &J);
    if (!(J > 0.0) && (rule == 0 || (m->energy == 0 && !(J < 0.0))))
        return NAN;
    return orc_W_of_psi0(s, beta_k, m->Dinf, m->D0);
}

/* dW/dF at a grid point (D entries): (1 - D(max(s, beta_k))) dpsi0/dF; NaN
 * where grid_W is excluded. */
static void grid_P(const orc_material *m, int32_t d, const double *F, double beta_k,
                   int32_t rule, double *P)
{
    int D = d * d;
    if (m->energy == 1) {
        if (d == 2) {
            orc_stress(m, F, beta_k, P);
        } else {
            for (int c = 0; c < D; ++c)
                P[c] = NAN;
        }
        return;
    }
    if (d == 2 && m->energy == 0 && rule == 0) {
        orc_stress(m, F, beta_k, P);
        return;
    }
    double J;
    double s = psi0_d(m, d, F, &J);
    int excluded = !(J > 0.0) && (rule == 0 || (m->energy == 0 && !(J < 0.0)));
    if (excluded) {
        for (int c = 0; c < D; ++c)
            P[c] = NAN;
        return;
    }
    double beta = s > beta_k ? s : beta_k;
    double gd = 1.0 - orc_damage(beta, m->Dinf, m->D0);
    double G[9];
    dpsi0_d(m, d, F, G);
    for (int c = 0; c < D; ++c)
        P[c] = gd * G[c];
}

/* d^2 W / dF dF at a grid point (D x D, A[D a + b] = dP_a / dF_b over the
 * row-major entries): with g = 1 - D(max(s, beta_k)) and, on loading
 * (s > beta_k), g' = -(D_inf / D_0) exp(-s / D_0),
 *   A = g d^2 psi0 + g' dpsi0 (x) dpsi0,
 *   Eq. (2.3), G = F^{-T}, ln|J|:
 *     d^2 psi0 / dF_iJ dF_kL = mu d_ik d_JL + lam G_iJ G_kL + (mu - lam ln|J|) G_iL G_kJ;
 *   Eq. (2.2), S = lam/2 (I1 - 3) 1 + mu (C - 1) (so dpsi0/dF = F S):
 *     d^2 psi0 / dF_iJ dF_kL = d_ik S_LJ + lam F_iJ F_kL + mu F_iL F_kJ + mu (F F^T)_ik d_JL.
 * NaN where grid_W is excluded; the double well through orc_tangent. */
static void grid_A(const orc_material *m, int32_t d, const double *F, double beta_k,
                   int32_t rule, double *A)
{
    int D = d * d;
    if (m->energy == 1) {
        if (d == 2) {
            orc_tangent(m, F, beta_k, A);
        } else {
            for (int c = 0; c < D * D; ++c)
                A[c] = NAN;
        }
        return;
    }
    double J;
    double s = psi0_d(m, d, F, &J);
    int excluded = !(J > 0.0) && (rule == 0 || (m->energy == 0 && !(J < 0.0)));
    if (excluded) {
        for (int c = 0; c < D * D; ++c)
            A[c] = NAN;
        return;
    }
    double beta = s > beta_k ? s : beta_k;
    double g = 1.0 - orc_damage(beta, m->Dinf, m->D0);
    double gp = s > beta_k ? -(m->Dinf / m->D0) * exp(-s / m->D0) : 0.0;
    double dp[9];
    dpsi0_d(m, d, F, dp);
    double I1, I2, JJ;
    orc_invariants(d, F, &I1, &I2, &JJ);
    double C[9], S[9], FFt[9], G[9];
    right_cauchy_green(d, F, C);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double v = 0.0;
            for (int k = 0; k < d; ++k)
                v += F[d * i + k] * F[d * j + k];
            FFt[d * i + j] = v;
            S[d * i + j] = m->mu * (C[d * i + j] - (i == j ? 1.0 : 0.0))
                         + (i == j ? 0.5 * m->lam * (I1 - 3.0) : 0.0);
        }
    double lj = 0.0;
    if (m->energy == 0) {
        double c[9];
        if (d == 2) {
            c[0] = F[3];
            c[1] = -F[2];
            c[2] = -F[1];
            c[3] = F[0];
        } else {
            cof3(F, c);
        }
        for (int k = 0; k < D; ++k)
            G[k] = c[k] / J;
        lj = log(fabs(J));
    }
    for (int i = 0; i < d; ++i)
        for (int Jc = 0; Jc < d; ++Jc)
            for (int k = 0; k < d; ++k)
                for (int L = 0; L < d; ++L) {
                    double d2;
                    if (m->energy == 2)
                        d2 = (i == k ? S[d * L + Jc] : 0.0) + m->lam * F[d * i + Jc] * F[d * k + L]
                           + m->mu * F[d * i + L] * F[d * k + Jc]
                           + (Jc == L ? m->mu * FFt[d * i + k] : 0.0);
                    else
                        d2 = (i == k && Jc == L ? m->mu : 0.0)
                           + m->lam * G[d * i + Jc] * G[d * k + L]
                           + (m->mu - m->lam * lj) * G[d * i + L] * G[d * k + Jc];
                    A[D * (d * i + Jc) + (d * k + L)] = g * d2 + gp * dp[d * i + Jc] * dp[d * k + L];
                }
}

void orc_tangent_dim(const orc_material *m, int32_t d, const double *F, double beta_k,
                     int32_t rule, double *A)
{
    grid_A(m, d, F, beta_k, rule, A);
}

/* W and P = dW/dF at one F in R^{d x d} under a grid rule (for tests). */
double orc_energy_dim(const orc_material *m, int32_t d, const double *F, double beta_k,
                      int32_t rule)
{
    return grid_W(m, d, F, beta_k, rule);
}

void orc_stress_dim(const orc_material *m, int32_t d, const double *F, double beta_k,
                    int32_t rule, double *P)
{
    grid_P(m, d, F, beta_k, rule, P);
}

/* W^0 on the grid: the energy at every grid point (NaN where it is not
 * defined). */
void orc_grid_energy(const orc_material *m, const orc_grid *g, double beta_k, int32_t rule,
                     double *W, int32_t nthreads)
{
    int64_t N = orc_grid_count(g);
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t idx = 0; idx < N; ++idx) {
        double F[9];
        orc_grid_point(g, idx, F);
        W[idx] = grid_W(m, g->dim, F, beta_k, rule);
    }
}

/* Range of steps l with grid index i + l off inside the grid. */
static void line_range(const orc_grid *g, const int32_t *i, const int32_t *off, int32_t *lo,
                       int32_t *hi)
{
    int32_t a = -(1 << 30), b = 1 << 30;
    for (int c = 0; c < grid_D(g); ++c) {
        if (off[c] > 0) {
            int32_t l0 = -i[c] / off[c], l1 = (g->n[c] - 1 - i[c]) / off[c];
            if (l0 > a) a = l0;
            if (l1 < b) b = l1;
        } else if (off[c] < 0) {
            int32_t l0 = -(g->n[c] - 1 - i[c]) / (-off[c]), l1 = i[c] / (-off[c]);
            if (l0 > a) a = l0;
            if (l1 < b) b = l1;
        }
    }
    *lo = a;
    *hi = b;
}

/* One global iteration, Eq. (4.3).  For every grid point F and direction R
 * (grid-index offset off[j], D entries): the values Win at the grid points
 * F + l R of the line through F inside the grid (Eq. 4.5; every point of the
 * line is a grid point, so no interpolation is needed), Algorithm 1 on the
 * finite ones (orc_line_bridge), read at l = 0.  Wout[F] = min(Win[F],
 * min_j h_j); the laminate is the lowest j with h_j < Win[F] at the minimum:
 * dir[F] = j and its bridge ends lm[F] < 0 < lp[F] (dir = -1, lm = lp = 0
 * otherwise).  Points where Win is not finite keep it.  hdir (N x nd, may be
 * NULL) receives every h_j.  Returns the largest decrease Win - Wout over the
 * points where both are finite. */
double orc_grid_step(const orc_grid *g, int32_t nd, const int32_t *off, const double *Win,
                     double *Wout, int32_t *dir, int32_t *lm, int32_t *lp, double *hdir,
                     int32_t nthreads)
{
    int64_t N = orc_grid_count(g);
    int D = grid_D(g);
    int32_t nmax = 0;
    for (int c = 0; c < D; ++c)
        if (g->n[c] > nmax)
            nmax = g->n[c];
    double dec = 0.0;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 256) reduction(max : dec)
#endif
    for (int64_t idx = 0; idx < N; ++idx) {
        int32_t i[9];
        grid_index(g, idx, i);
        double w0 = Win[idx];
        int32_t bj = -1, bm = 0, bp = 0;
        double best = w0;
        int32_t L = 2 * nmax + 1, M = nmax;
        double *w = (double *)malloc(sizeof(double) * L);
        uint8_t *valid = (uint8_t *)malloc(L);
        for (int32_t j = 0; j < nd; ++j) {
            const int32_t *o = off + D * j;
            double h = w0;
            if (isfinite(w0)) {
                int32_t l0, l1;
                line_range(g, i, o, &l0, &l1);
                for (int32_t m = 0; m < L; ++m) {
                    int32_t l = m - M;
                    valid[m] = 0;
                    w[m] = 0.0;
                    if (l < l0 || l > l1)
                        continue;
                    int32_t ii[9];
                    for (int c = 0; c < D; ++c)
                        ii[c] = i[c] + l * o[c];
                    double v = Win[grid_flat(g, ii)];
                    if (isfinite(v)) {
                        w[m] = v;
                        valid[m] = 1;
                    }
                }
                int32_t mm, mp;
                h = orc_line_bridge(L, w, valid, &mm, &mp, NULL);
                if (mm != M && h < best) {
                    best = h;
                    bj = j;
                    bm = mm - M;
                    bp = mp - M;
                }
            }
            if (hdir)
                hdir[idx * nd + j] = h;
        }
        free(w);
        free(valid);
        Wout[idx] = best;
        if (dir) {
            dir[idx] = bj;
            lm[idx] = bm;
            lp[idx] = bp;
        }
        if (isfinite(w0) && isfinite(best) && w0 - best > dec)
            dec = w0 - best;
    }
    return dec;
}

/* Interpolation decomposition of F (Sec. 5.3, Algorithm 2): the corners of
 * the grid cell that contains F and their multilinear weights
 * prod_c (1 - t_c or t_c), t_c = (F_c - lo_c) / delta_c - i_c; a t_c within
 * 1e-12 of 0 or 1 counts as 0 or 1, so that a grid point is its own single
 * corner; corners of weight 0 are left out (2^D candidates, corner bit c of
 * the corner number counted from the first component).  Returns the number
 * of corners, 0 if F lies outside the grid. */
static int32_t grid_decompose(const orc_grid *g, const double *F, int64_t *cidx, double *cw)
{
    int D = grid_D(g);
    int32_t i0[9];
    double t[9];
    for (int c = 0; c < D; ++c) {
        double u = (F[c] - g->lo[c]) / g->delta[c];
        if (u < -1e-12 || u > (double)(g->n[c] - 1) + 1e-12)
            return 0;
        double f = floor(u);
        double r = u - f;
        if (r > 1.0 - 1e-12) {
            f += 1.0;
            r = 0.0;
        } else if (r < 1e-12) {
            r = 0.0;
        }
        int32_t ii = (int32_t)f;
        if (ii > g->n[c] - 1)
            ii = g->n[c] - 1;
        if (ii < 0)
            ii = 0;
        i0[c] = ii;
        t[c] = r;
    }
    int32_t nc = 0;
    for (int corner = 0; corner < (1 << D); ++corner) {
        double w = 1.0;
        int32_t ii[9];
        for (int c = 0; c < D; ++c) {
            int up = (corner >> (D - 1 - c)) & 1;
            w *= up ? t[c] : 1.0 - t[c];
            ii[c] = i0[c] + up;
        }
        if (w == 0.0)
            continue;
        cidx[nc] = grid_flat(g, ii);
        cw[nc] = w;
        ++nc;
    }
    return nc;
}

/* Algorithm 2's tree below grid point idx at order d, evaluated by
 * Algorithm 3: the laminate of the latest iteration k <= d that split idx
 * (forest[k - 1]) gives the children F-+ = F + l-+ R at order k - 1 with
 * weights 1 - xi and xi, xi = -l- / (l+ - l-) (Algorithm 2's
 * |F - F-|_1 / |F+ - F-|_1); a point no iteration up to d split is a leaf,
 * where W and P are evaluated.  Adds weight * (W, P) of the leaves. */
static void grid_tree(const orc_material *mat, const orc_grid *g, double beta_k, int32_t rule,
                      const int32_t *off, const int32_t *forest, int64_t idx, int32_t d,
                      double weight, double *W, double *P, double *A, int64_t *leaves)
{
    int64_t N = orc_grid_count(g);
    int D = grid_D(g);
    int32_t k = d;
    while (k >= 1 && forest[3 * ((int64_t)(k - 1) * N + idx)] < 0)
        --k;
    if (k < 1) {
        double F[9], Pl[9];
        orc_grid_point(g, idx, F);
        *W += weight * grid_W(mat, g->dim, F, beta_k, rule);
        grid_P(mat, g->dim, F, beta_k, rule, Pl);
        for (int c = 0; c < D; ++c)
            P[c] += weight * Pl[c];
        if (A) {
            double Al[81];
            grid_A(mat, g->dim, F, beta_k, rule, Al);
            for (int c = 0; c < D * D; ++c)
                A[c] += weight * Al[c];
        }
        ++*leaves;
        return;
    }
    const int32_t *lam = forest + 3 * ((int64_t)(k - 1) * N + idx);
    const int32_t *o = off + D * lam[0];
    int32_t lm = lam[1], lp = lam[2];
    double xi = (double)(-lm) / (double)(lp - lm);
    int32_t i[9], im[9], ip[9];
    grid_index(g, idx, i);
    for (int c = 0; c < D; ++c) {
        im[c] = i[c] + lm * o[c];
        ip[c] = i[c] + lp * o[c];
    }
    grid_tree(mat, g, beta_k, rule, off, forest, grid_flat(g, im), k - 1, weight * (1.0 - xi), W,
              P, A, leaves);
    grid_tree(mat, g, beta_k, rule, off, forest, grid_flat(g, ip), k - 1, weight * xi, W, P, A,
              leaves);
}

/* Relaxed energy, stress and tangent at arbitrary points from K global
 * iterations (A: n x D^2, nullable; Algorithm 3's third output):
 * W_interp = the multilinear interpolation of W^K (Sec. 4.1: values off the
 * grid by interpolation); W_tree, P = Algorithm 3 over Algorithm 2's tree
 * (the interpolation corners at order K, then the forest).  F and P hold D
 * entries per point; forest holds K x N records (dir, l-, l+) (dir = -1: no
 * split).  leaves[p] counts the tree's leaves.  Outside the grid: NaN,
 * leaves 0. */
void orc_grid_query(const orc_material *mat, const orc_grid *g, double beta_k, int32_t rule,
                    const int32_t *off, int32_t K, const double *WK, const int32_t *forest,
                    int64_t n, const double *F, double *W_interp, double *W_tree, double *P,
                    double *A, int64_t *leaves, int32_t nthreads)
{
    int D = grid_D(g);
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < n; ++p) {
        int64_t *cidx = (int64_t *)malloc(sizeof(int64_t) << D);
        double *cw = (double *)malloc(sizeof(double) << D);
        int32_t nc = grid_decompose(g, F + D * p, cidx, cw);
        double wi = 0.0, wt = 0.0, Pp[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double *Ap = A ? A + (int64_t)D * D * p : NULL;
        if (Ap)
            for (int c = 0; c < D * D; ++c)
                Ap[c] = 0.0;
        int64_t nl = 0;
        for (int32_t c = 0; c < nc; ++c) {
            wi += cw[c] * WK[cidx[c]];
            grid_tree(mat, g, beta_k, rule, off, forest, cidx[c], K, cw[c], &wt, Pp, Ap, &nl);
        }
        if (nc == 0) {
            wi = wt = NAN;
            for (int c = 0; c < D; ++c)
                Pp[c] = NAN;
            if (Ap)
                for (int c = 0; c < D * D; ++c)
                    Ap[c] = NAN;
        }
        W_interp[p] = wi;
        W_tree[p] = wt;
        for (int c = 0; c < D; ++c)
            P[D * p + c] = Pp[c];
        leaves[p] = nl;
        free(cidx);
        free(cw);
    }
}
