/*
 * FP64 CPU oracle for the DMTS-NC hot path. TEST INFRASTRUCTURE ONLY: it is
 * loaded by the tests, by the smoke check and by the CPU-baseline leg of the
 * benchmark, never by the product path. It shares no code with the CUDA
 * library; both read the same seeded inputs.
 *
 * Everything is written as plain loops in the order the definitions state:
 * no blocking, no fusion, no reordering. Units: A, fs, amu, kcal/mol, K.
 *
 * Contents (paper sections / equations each function follows):
 *   orc_nbr_brute     neighbour set N(i): all j != i within the cutoff, with the
 *                     minimum-image convention (Sec. 2 "Model architecture",
 *                     Sec. 2 "virial term" for minimum image).
 *   orc_cons_*        conservative message-passing energy U and F = -grad U
 *                     (Sec. 2 "Model architecture": embedding + message passing;
 *                     Sec. 2 "Multi-time-step integrator": F = -grad U). The
 *                     exact model is a stand-in (trained weights are not
 *                     available): parity of its absolute value with the paper's
 *                     FeNNix-Bio1(M) is unpinned by design; it is pinned by
 *                     finite differences and invariances.
 *   orc_nc_forces     non-conservative direct forces: q/k projections, scaled
 *                     dot products c_ijh, Bessel radial basis, polynomial
 *                     cutoff, pair forces F_ij, antisymmetric sum F_i, plus the
 *                     mean-force subtraction (Sec. 2 "Model architecture").
 *   orc_prior         analytic terms: harmonic bonds, Lennard-Jones between heavy
 *                     atoms of different molecules, and the screened nuclear
 *                     repulsion E_rep of Sec. 2 (ZBL universal screening standing
 *                     in for the NHL pair parameters, which are not given).
 *   orc_philox4x32_10 / orc_gauss3   counter-based noise (Salmon et al., SC'11).
 *   orc_hmr_masses    hydrogen mass repartitioning (Sec. 2 "HMR").
 *   orc_gamma_table   per-species Langevin O-step constants (Sec. 2 "HHF";
 *                     BAOAB O-step of Leimkuhler & Matthews).
 *   orc_respa_run     Algorithm 1 (DMTS-NC integration step), force caching
 *                     across outer steps.
 *   orc_sts_run       single-time-step BAOAB (Sec. 2, Sec. 3 setup).
 *   orc_respa_run with a barostat: isotropic Langevin piston around the outer
 *                     step, driven by the virial estimator of Sec. 2
 *                     "Computation of the virial term in NPT" (Sec. 3: Bussi's
 *                     barostat, 1 atm, tau_P = 2 ps); the scheme is the reading
 *                     stated at orc_baro_* below.
 *   Both take the O-step's thermostat: Langevin, or the Fast Forward Langevin
 *   update of Sec. 2 "High Hydrogen Friction" (the Langevin speed, the old
 *   direction, per-atom norms).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SP_H 0
#define ORC_MAX_LAYERS 8
#define ORC_ACC_CONV 4.184e-4                 /* (kcal/mol/A)/amu -> A/fs^2 */
#define ORC_KB (8.314462618 / 4184.0)         /* kcal/mol/K */

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Minimum-image displacement d = x_j - x_i on periodic axes (box[a] > 0). */
static void min_image(const double *xi, const double *xj, const double *box, double *d)
{
    for (int a = 0; a < 3; ++a) {
        double t = xj[a] - xi[a];
        if (box[a] > 0.0) t -= box[a] * rint(t / box[a]);
        d[a] = t;
    }
}

/* Full (both-direction) neighbour list by brute force: j in row i iff j != i
 * and |d_ij|^2 < rcut^2 (strict). Rows ascend in j. Returns the number of
 * pairs, or -(needed) when cap is too small. */
long orc_nbr_brute(int n, const double *x, const double *box, double rcut,
                   int *row_ptr, int *col, long cap)
{
    long e = 0;
    double r2 = rcut * rcut;
    for (int i = 0; i < n; ++i) {
        row_ptr[i] = (int)(e < cap ? e : cap);
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], box, d);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < r2) {
                if (e < cap) col[e] = j;
                ++e;
            }
        }
    }
    row_ptr[n] = (int)(e < cap ? e : cap);
    return e <= cap ? e : -e;
}

/* Edge set used by the models: directed pairs (i, j) with r < rc. */
typedef struct {
    long n;
    int *i, *j;
    double *d;   /* [n][3] displacement x_j - x_i */
    double *r;
} edges_t;

static void edges_build(int n_atoms, const double *x, const double *box, double rc, edges_t *E)
{
    long cap = 64, n = 0;
    E->i = malloc(cap * sizeof(int));
    E->j = malloc(cap * sizeof(int));
    E->d = malloc(cap * 3 * sizeof(double));
    E->r = malloc(cap * sizeof(double));
    for (int i = 0; i < n_atoms; ++i)
        for (int j = 0; j < n_atoms; ++j) {
            if (j == i) continue;
            double d[3];
            min_image(&x[3 * i], &x[3 * j], box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            if (n == cap) {
                cap *= 2;
                E->i = realloc(E->i, cap * sizeof(int));
                E->j = realloc(E->j, cap * sizeof(int));
                E->d = realloc(E->d, cap * 3 * sizeof(double));
                E->r = realloc(E->r, cap * sizeof(double));
            }
            E->i[n] = i;
            E->j[n] = j;
            E->d[3 * n] = d[0];
            E->d[3 * n + 1] = d[1];
            E->d[3 * n + 2] = d[2];
            E->r[n] = sqrt(r2);
            ++n;
        }
    E->n = n;
}

static void edges_free(edges_t *E)
{
    free(E->i); free(E->j); free(E->d); free(E->r);
}

/* ------------------------------------------------------------------------ */
/* Radial basis, envelope, spherical harmonics                               */
/* ------------------------------------------------------------------------ */

/* Bessel radial basis of Gasteiger et al. (DimeNet), k = 1..K:
 * B_k(r) = sqrt(2/rc) sin(k pi r / rc) / r, and its r-derivative. */
double orc_bessel(int k, double r, double rc)
{
    return sqrt(2.0 / rc) * sin(k * M_PI * r / rc) / r;
}

double orc_dbessel(int k, double r, double rc)
{
    double w = k * M_PI / rc;
    return sqrt(2.0 / rc) * (w * cos(w * r) / r - sin(w * r) / (r * r));
}

/* Polynomial cutoff of Gasteiger et al. with exponent p, u = r/rc < 1:
 * f(u) = 1 - (p+1)(p+2)/2 u^p + p(p+2) u^(p+1) - p(p+1)/2 u^(p+2). */
double orc_envelope(double u, double p)
{
    if (u >= 1.0) return 0.0;
    return 1.0 - (p + 1) * (p + 2) / 2.0 * pow(u, p) + p * (p + 2) * pow(u, p + 1)
           - p * (p + 1) / 2.0 * pow(u, p + 2);
}

double orc_denvelope(double u, double p)
{
    if (u >= 1.0) return 0.0;
    return -p * (p + 1) * (p + 2) / 2.0 * pow(u, p - 1) + p * (p + 1) * (p + 2) * pow(u, p)
           - p * (p + 1) * (p + 2) / 2.0 * pow(u, p + 1);
}

/* Real spherical harmonics, component normalisation (sum_m Y_lm^2 = 2l+1),
 * of the unit vector n, l <= 2, in the order
 * [Y00 | Y1x Y1y Y1z | xy yz (3z^2-1) xz (x^2-y^2)]. */
void orc_sph(const double *n, double *Y)
{
    const double s3 = sqrt(3.0), s5 = sqrt(5.0), s15 = sqrt(15.0);
    double x = n[0], y = n[1], z = n[2];
    Y[0] = 1.0;
    Y[1] = s3 * x; Y[2] = s3 * y; Y[3] = s3 * z;
    Y[4] = s15 * x * y;
    Y[5] = s15 * y * z;
    Y[6] = 0.5 * s5 * (3.0 * z * z - 1.0);
    Y[7] = s15 * x * z;
    Y[8] = 0.5 * s15 * (x * x - y * y);
}

/* Gradient of Y_lm(d/|d|) with respect to the displacement d:
 * dY/dd = (I - n n^T) (grad_n Y) / r. dY[lm][a]. */
static void sph_grad(const double *n, double r, double *dY)
{
    const double s3 = sqrt(3.0), s5 = sqrt(5.0), s15 = sqrt(15.0);
    double x = n[0], y = n[1], z = n[2];
    double g[9][3] = {
        {0, 0, 0},
        {s3, 0, 0}, {0, s3, 0}, {0, 0, s3},
        {s15 * y, s15 * x, 0},
        {0, s15 * z, s15 * y},
        {0, 0, 3.0 * s5 * z},
        {s15 * z, 0, s15 * x},
        {s15 * x, -s15 * y, 0},
    };
    for (int lm = 0; lm < 9; ++lm) {
        double ng = n[0] * g[lm][0] + n[1] * g[lm][1] + n[2] * g[lm][2];
        for (int a = 0; a < 3; ++a) dY[3 * lm + a] = (g[lm][a] - n[a] * ng) / r;
    }
}

static double silu(double v) { return v / (1.0 + exp(-v)); }
static double dsilu(double v)
{
    double sg = 1.0 / (1.0 + exp(-v));
    return sg * (1.0 + v * (1.0 - sg));
}

/* Screened nuclear repulsion standing in for the NHL term of Sec. 2 (whose
 * pair parameters are not given): E_rep = k_e Z_i Z_j / r * phi(r/a) with
 * the universal screening function of Ziegler, Biersack and Littmark (1985),
 * phi(x) = sum_k c_k exp(-d_k x), a = 0.8854 a_0 / (Z_i^0.23 + Z_j^0.23),
 * switched off by the envelope f(r/rc; p). Returns E and dE/dr. */
static const double ORC_ZBL_C[4] = {0.18175, 0.50986, 0.28022, 0.02817};
static const double ORC_ZBL_D[4] = {3.19980, 0.94229, 0.40290, 0.20162};
static const double ORC_Z[5] = {1.0, 6.0, 7.0, 8.0, 16.0};     /* H C N O S */
#define ORC_KE 332.0637133       /* e^2/(4 pi eps0) in kcal/mol * A */
#define ORC_A0 0.529177210903    /* Bohr radius, A */

double orc_zbl_phi(double x)
{
    double s = 0.0;
    for (int k = 0; k < 4; ++k) s += ORC_ZBL_C[k] * exp(-ORC_ZBL_D[k] * x);
    return s;
}

double orc_rep_pair(int si, int sj, double r, double rc, double p, double *dEdr)
{
    double zi = ORC_Z[si], zj = ORC_Z[sj];
    double a = 0.8854 * ORC_A0 / (pow(zi, 0.23) + pow(zj, 0.23));
    double x = r / a, phi = 0.0, dphi = 0.0;
    for (int k = 0; k < 4; ++k) {
        double t = ORC_ZBL_C[k] * exp(-ORC_ZBL_D[k] * x);
        phi += t;
        dphi -= ORC_ZBL_D[k] * t;
    }
    double u = r / rc, fc = orc_envelope(u, p), dfc = orc_denvelope(u, p) / rc;
    double c = ORC_KE * zi * zj;
    double e0 = c / r * phi;
    double de0 = -c / (r * r) * phi + c / r * dphi / a;
    if (dEdr) *dEdr = de0 * fc + e0 * dfc;
    return e0 * fc;
}

static int l_of(int lm) { return lm == 0 ? 0 : (lm < 4 ? 1 : 2); }

/* ------------------------------------------------------------------------ */
/* Model parameters                                                          */
/* ------------------------------------------------------------------------ */

/* ints: [L, C, lmax, K, n_species, n_c, n_l]; reals: [rc, p, nu, scale] */
typedef struct {
    int L, C, lmax, K, S, nc, nl, nlm;
    double rc, p, nu, scale;
    const double *emb;
    const double *wrad[ORC_MAX_LAYERS], *w1[ORC_MAX_LAYERS], *b1[ORC_MAX_LAYERS],
        *w2[ORC_MAX_LAYERS], *b2[ORC_MAX_LAYERS];
    const double *wr, *br, *wo;      /* conservative readout */
    const double *U, *Wq, *Wk;       /* NC head */
} model_t;

static void model_common(model_t *m, const int *mi, const double *mr)
{
    m->L = mi[0]; m->C = mi[1]; m->lmax = mi[2]; m->K = mi[3]; m->S = mi[4];
    m->nc = mi[5]; m->nl = mi[6];
    m->nlm = (m->lmax + 1) * (m->lmax + 1);
    m->rc = mr[0]; m->p = mr[1]; m->nu = mr[2]; m->scale = mr[3];
}

/* Conservative blob: emb[S][C]; per layer wrad[lmax+1][K][C], w1[C][(lmax+1)C],
 * b1[C], w2[C][C], b2[C]; then wr[C][C], br[C], wo[C]. */
static void parse_cons(model_t *m, const int *mi, const double *mr, const double *w)
{
    model_common(m, mi, mr);
    int C = m->C, K = m->K, nl1 = m->lmax + 1;
    m->emb = w; w += m->S * C;
    for (int t = 0; t < m->L; ++t) {
        m->wrad[t] = w; w += nl1 * K * C;
        m->w1[t] = w; w += C * nl1 * C;
        m->b1[t] = w; w += C;
        m->w2[t] = w; w += C * C;
        m->b2[t] = w; w += C;
    }
    m->wr = w; w += C * C;
    m->br = w; w += C;
    m->wo = w;
}

/* NC blob: emb[S][C]; wrad[2][K][C], w1[C][2C], b1[C], w2[C][C], b2[C];
 * U[n_l][C]; Wq[H][n_c][C]; Wk[H][n_c][C], H = K + n_l. */
static void parse_nc(model_t *m, const int *mi, const double *mr, const double *w)
{
    model_common(m, mi, mr);
    int C = m->C, K = m->K, H = m->K + m->nl;
    m->L = 1;
    m->emb = w; w += m->S * C;
    m->wrad[0] = w; w += 2 * K * C;
    m->w1[0] = w; w += C * 2 * C;
    m->b1[0] = w; w += C;
    m->w2[0] = w; w += C * C;
    m->b2[0] = w; w += C;
    m->U = w; w += m->nl * C;
    m->Wq = w; w += H * m->nc * C;
    m->Wk = w;
}

/* ------------------------------------------------------------------------ */
/* Message-passing layer (shared definition of both models' embedding)       */
/* ------------------------------------------------------------------------ */

/* One layer t: A_i[c][lm] = nu * sum_{j in N(i)} R_lc(r_ij) s_j[c] Y_lm(n_ij),
 * R_lc(r) = f(r/rc) * sum_k wrad[l][k][c] B_k(r);
 * q_i[l*C + c] = sum_{m} A_i[c][lm]^2;
 * h_i = W1 q_i + b1;  s_i' = s_i + W2 silu(h_i) + b2. */
static void mp_layer_forward(const model_t *m, int t, int n, const edges_t *E,
                             const double *s, double *A, double *q, double *h, double *s_out)
{
    int C = m->C, K = m->K, nlm = m->nlm, nl1 = m->lmax + 1;
    memset(A, 0, sizeof(double) * n * C * nlm);
    for (long e = 0; e < E->n; ++e) {
        int i = E->i[e], j = E->j[e];
        double r = E->r[e], nvec[3], Y[9];
        for (int a = 0; a < 3; ++a) nvec[a] = E->d[3 * e + a] / r;
        orc_sph(nvec, Y);
        double fc = orc_envelope(r / m->rc, m->p);
        double B[64];
        for (int k = 0; k < K; ++k) B[k] = orc_bessel(k + 1, r, m->rc);
        for (int c = 0; c < C; ++c)
            for (int l = 0; l < nl1; ++l) {
                double R = 0.0;
                for (int k = 0; k < K; ++k) R += m->wrad[t][(l * K + k) * C + c] * B[k];
                R *= fc;
                for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm)
                    A[((long)i * C + c) * nlm + lm] += m->nu * R * s[(long)j * C + c] * Y[lm];
            }
    }
    for (int i = 0; i < n; ++i) {
        for (int l = 0; l < nl1; ++l)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int lm = 0; lm < nlm; ++lm)
                    if (l_of(lm) == l) {
                        double a = A[((long)i * C + c) * nlm + lm];
                        acc += a * a;
                    }
                q[(long)i * nl1 * C + l * C + c] = acc;
            }
        for (int o = 0; o < C; ++o) {
            double acc = m->b1[t][o];
            for (int in = 0; in < nl1 * C; ++in)
                acc += m->w1[t][o * nl1 * C + in] * q[(long)i * nl1 * C + in];
            h[(long)i * C + o] = acc;
        }
        for (int c = 0; c < C; ++c) {
            double acc = m->b2[t][c];
            for (int o = 0; o < C; ++o) acc += m->w2[t][c * C + o] * silu(h[(long)i * C + o]);
            s_out[(long)i * C + c] = s[(long)i * C + c] + acc;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Conservative model: energy and analytic forces                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    const double *x;
    const uint8_t *species;
    const double *box;
} sys_t;

/* U_MP = scale * sum_i sum_o wo[o] silu((Wr s_i^L + br)[o]); optional forces
 * F = -dU_MP/dx by reverse-mode differentiation of every step above. */
static double cons_eval(const model_t *m, const sys_t *sy, double *e_atom, double *F)
{
    int n = sy->n, C = m->C, L = m->L, nlm = m->nlm, nl1 = m->lmax + 1, K = m->K;
    edges_t E;
    edges_build(n, sy->x, sy->box, m->rc, &E);
    double **s = malloc(sizeof(double *) * (L + 1));
    double **A = malloc(sizeof(double *) * L);
    double **q = malloc(sizeof(double *) * L);
    double **h = malloc(sizeof(double *) * L);
    for (int t = 0; t <= L; ++t) s[t] = malloc(sizeof(double) * n * C);
    for (int t = 0; t < L; ++t) {
        A[t] = malloc(sizeof(double) * n * C * nlm);
        q[t] = malloc(sizeof(double) * n * nl1 * C);
        h[t] = malloc(sizeof(double) * n * C);
    }
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < C; ++c) s[0][(long)i * C + c] = m->emb[sy->species[i] * C + c];
    for (int t = 0; t < L; ++t) mp_layer_forward(m, t, n, &E, s[t], A[t], q[t], h[t], s[t + 1]);

    double *z = malloc(sizeof(double) * n * C);
    double energy = 0.0;
    for (int i = 0; i < n; ++i) {
        double ei = 0.0;
        for (int o = 0; o < C; ++o) {
            double acc = m->br[o];
            for (int c = 0; c < C; ++c) acc += m->wr[o * C + c] * s[L][(long)i * C + c];
            z[(long)i * C + o] = acc;
            ei += m->wo[o] * silu(acc);
        }
        if (e_atom) e_atom[i] = m->scale * ei;
        energy += m->scale * ei;
    }

    if (F) {
        for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
        double *gs = malloc(sizeof(double) * n * C);
        double *gs_new = malloc(sizeof(double) * n * C);
        double *gh = malloc(sizeof(double) * n * C);
        double *gq = malloc(sizeof(double) * n * nl1 * C);
        double *gA = malloc(sizeof(double) * n * C * nlm);
        /* dU/ds^L */
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < C; ++c) {
                double acc = 0.0;
                for (int o = 0; o < C; ++o)
                    acc += m->wo[o] * dsilu(z[(long)i * C + o]) * m->wr[o * C + c];
                gs[(long)i * C + c] = m->scale * acc;
            }
        for (int t = L - 1; t >= 0; --t) {
            for (int i = 0; i < n; ++i) {
                for (int o = 0; o < C; ++o) {
                    double acc = 0.0;
                    for (int c = 0; c < C; ++c) acc += m->w2[t][c * C + o] * gs[(long)i * C + c];
                    gh[(long)i * C + o] = dsilu(h[t][(long)i * C + o]) * acc;
                }
                for (int in = 0; in < nl1 * C; ++in) {
                    double acc = 0.0;
                    for (int o = 0; o < C; ++o) acc += m->w1[t][o * nl1 * C + in] * gh[(long)i * C + o];
                    gq[(long)i * nl1 * C + in] = acc;
                }
                for (int c = 0; c < C; ++c)
                    for (int lm = 0; lm < nlm; ++lm)
                        gA[((long)i * C + c) * nlm + lm] =
                            2.0 * A[t][((long)i * C + c) * nlm + lm] * gq[(long)i * nl1 * C + l_of(lm) * C + c];
            }
            memcpy(gs_new, gs, sizeof(double) * n * C);   /* identity (residual) path */
            for (long e = 0; e < E.n; ++e) {
                int i = E.i[e], j = E.j[e];
                double r = E.r[e], nvec[3], Y[9], dY[27], gd[3] = {0, 0, 0};
                for (int a = 0; a < 3; ++a) nvec[a] = E.d[3 * e + a] / r;
                orc_sph(nvec, Y);
                sph_grad(nvec, r, dY);
                double u = r / m->rc;
                double fc = orc_envelope(u, m->p), dfc = orc_denvelope(u, m->p) / m->rc;
                double B[64], dB[64];
                for (int k = 0; k < K; ++k) {
                    B[k] = orc_bessel(k + 1, r, m->rc);
                    dB[k] = orc_dbessel(k + 1, r, m->rc);
                }
                for (int c = 0; c < C; ++c)
                    for (int l = 0; l < nl1; ++l) {
                        double sb = 0.0, sdb = 0.0;
                        for (int k = 0; k < K; ++k) {
                            double w = m->wrad[t][(l * K + k) * C + c];
                            sb += w * B[k];
                            sdb += w * dB[k];
                        }
                        double R = fc * sb, dR = dfc * sb + fc * sdb;   /* R_lc and dR_lc/dr */
                        double sj = s[t][(long)j * C + c];
                        for (int lm = l * l; lm < (l + 1) * (l + 1); ++lm) {
                            double g = m->nu * gA[((long)i * C + c) * nlm + lm];
                            gs_new[(long)j * C + c] += g * R * Y[lm];
                            for (int a = 0; a < 3; ++a)
                                gd[a] += g * sj * (dR * Y[lm] * nvec[a] + R * dY[3 * lm + a]);
                        }
                    }
                /* d = x_j - x_i: F_i = -dU/dx_i = +dU/dd, F_j = -dU/dd */
                for (int a = 0; a < 3; ++a) {
                    F[3 * i + a] += gd[a];
                    F[3 * j + a] -= gd[a];
                }
            }
            memcpy(gs, gs_new, sizeof(double) * n * C);
        }
        free(gs); free(gs_new); free(gh); free(gq); free(gA);
    }
    free(z);
    for (int t = 0; t <= L; ++t) free(s[t]);
    for (int t = 0; t < L; ++t) { free(A[t]); free(q[t]); free(h[t]); }
    free(s); free(A); free(q); free(h);
    edges_free(&E);
    return energy;
}

double orc_cons_energy(int n, const double *x, const uint8_t *species, const double *box,
                       const int *mi, const double *mr, const double *blob, double *e_atom)
{
    model_t m;
    parse_cons(&m, mi, mr, blob);
    sys_t sy = {n, x, species, box};
    return cons_eval(&m, &sy, e_atom, NULL);
}

double orc_cons_energy_forces(int n, const double *x, const uint8_t *species, const double *box,
                              const int *mi, const double *mr, const double *blob, double *F)
{
    model_t m;
    parse_cons(&m, mi, mr, blob);
    sys_t sy = {n, x, species, box};
    return cons_eval(&m, &sy, NULL, F);
}

/* ------------------------------------------------------------------------ */
/* Prior: harmonic bonds + Lennard-Jones between heavy atoms of different    */
/* molecules, switched off smoothly at 5 A by the p=6 envelope.              */
/* ------------------------------------------------------------------------ */

/* Per-atom bond partners (CSR) for the bonded-pair exclusion. */
static void bond_adjacency(int n, int n_bonds, const int *bonds, int **ptr_out, int **idx_out)
{
    int *ptr = calloc(n + 1, sizeof(int));
    int *idx = malloc(sizeof(int) * (2 * n_bonds + 1));
    for (int b = 0; b < n_bonds; ++b) {
        ptr[bonds[2 * b] + 1]++;
        ptr[bonds[2 * b + 1] + 1]++;
    }
    for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    int *fill = malloc(sizeof(int) * (n + 1));
    memcpy(fill, ptr, sizeof(int) * (n + 1));
    for (int b = 0; b < n_bonds; ++b) {
        idx[fill[bonds[2 * b]]++] = bonds[2 * b + 1];
        idx[fill[bonds[2 * b + 1]]++] = bonds[2 * b];
    }
    free(fill);
    *ptr_out = ptr;
    *idx_out = idx;
}

/* reals: [k_bond, lj_eps, lj_sigma, lj_rc, lj_p, rep_rc, rep_p].
 * terms: bit 0 bonds, bit 1 LJ, bit 2 screened repulsion (all pairs i < j
 * closer than rep_rc that are not bonded). */
double orc_prior(int n, const double *x, const uint8_t *species, const int *mol_id,
                 const double *box, int n_bonds, const int *bonds, const double *bond_r0,
                 const double *pr, int terms, double *F, double *virial)
{
    /* virial (nullable): -sum_i F_i . q_i written with pair terms, the sum
     * over pairs of r dE/dr (Sec. 2 "Computation of the virial term in NPT") */
    if (virial) *virial = 0.0;
    double kb = pr[0], eps = pr[1], sig = pr[2], rlj = pr[3], plj = pr[4];
    double rrep = pr[5], prep = pr[6];
    int with_lj = (terms & 2) != 0;
    double E = 0.0;
    if (F) for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    for (int b = 0; (terms & 1) && b < n_bonds; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        min_image(&x[3 * i], &x[3 * j], box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dr = r - bond_r0[b];
        E += 0.5 * kb * dr * dr;
        if (virial) *virial += kb * dr * r;
        if (F) {
            double g = kb * dr / r;   /* dE/dd = g d */
            for (int a = 0; a < 3; ++a) {
                F[3 * i + a] += g * d[a];
                F[3 * j + a] -= g * d[a];
            }
        }
    }
    if (with_lj) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                if (species[i] == ORC_SP_H || species[j] == ORC_SP_H) continue;
                if (mol_id[i] == mol_id[j]) continue;
                double d[3];
                min_image(&x[3 * i], &x[3 * j], box, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rlj * rlj)) continue;
                double r = sqrt(r2);
                double sr6 = pow(sig / r, 6.0);
                double elj = 4.0 * eps * (sr6 * sr6 - sr6);
                double delj = 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
                double u = r / rlj;
                double fc = orc_envelope(u, plj), dfc = orc_denvelope(u, plj) / rlj;
                E += elj * fc;
                if (virial) *virial += (delj * fc + elj * dfc) * r;
                if (F) {
                    double g = (delj * fc + elj * dfc) / r;
                    for (int a = 0; a < 3; ++a) {
                        F[3 * i + a] += g * d[a];
                        F[3 * j + a] -= g * d[a];
                    }
                }
            }
    }
    if (terms & 4) {
        int *bp, *bi;
        bond_adjacency(n, n_bonds, bonds, &bp, &bi);
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double d[3];
                min_image(&x[3 * i], &x[3 * j], box, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < rrep * rrep)) continue;
                int is_bonded = 0;
                for (int q = bp[i]; q < bp[i + 1]; ++q) is_bonded |= bi[q] == j;
                if (is_bonded) continue;
                double r = sqrt(r2), dEdr;
                E += orc_rep_pair(species[i], species[j], r, rrep, prep, &dEdr);
                if (virial) *virial += dEdr * r;
                if (F) {
                    double g = dEdr / r;
                    for (int a = 0; a < 3; ++a) {
                        F[3 * i + a] += g * d[a];
                        F[3 * j + a] -= g * d[a];
                    }
                }
            }
        free(bp);
        free(bi);
    }
    return E;
}

/* ------------------------------------------------------------------------ */
/* Non-conservative direct-force model                                       */
/* ------------------------------------------------------------------------ */

/* Embedding: one message-passing layer (l_max = 1, short-range cutoff) gives
 * x_i = s_i^1 and the tensor embedding A_i[c][l=1][:].
 * V_ih = sum_c U[h][c] A_i[c][1,:] (vector part of tensor head h).
 * q_ih = Wq_h x_i, k_ih = Wk_h x_i in R^{n_c}.
 * c_ijh = (1/sqrt(n_c)) sum_k q_ihk k_jhk.
 * F_ij = (sum_{h<n_s} c_ijh B_h(r)) (R_ij/r + sum_{h<n_l} c_ij(n_s+h) V_ih) f_c(r).
 * F_i = scale * sum_{j in N(i)} (F_ij - F_ji); the fast prior terms selected
 * by fast_terms (bit 0 bonds, bit 2 screened repulsion F_rep) are added; then
 * the FP64 mean (sum_i F_i / N) is subtracted.
 * net_pre (optional, 3 doubles) receives sum_i F_i before subtraction. */
void orc_nc_forces(int n, const double *x, const uint8_t *species, const double *box,
                   const int *mi, const double *mr, const double *blob,
                   int n_bonds, const int *bonds, const double *bond_r0, const double *pr,
                   int fast_terms, double *F, double *net_pre, double *virial)
{
    /* virial (nullable): the proxy -sum_i F_i . q_i of Sec. 2 "Computation of
     * the virial term in NPT", as sum_i sum_{j in N(i)} F_ij . r_ij (scaled
     * like the forces) plus the pair form of the fast analytic terms */
    double W = 0.0;
    model_t m;
    parse_nc(&m, mi, mr, blob);
    int C = m.C, K = m.K, nl = m.nl, nc = m.nc, H = K + nl, nlm = m.nlm;
    edges_t E;
    edges_build(n, x, box, m.rc, &E);
    double *s0 = malloc(sizeof(double) * n * C);
    double *s1 = malloc(sizeof(double) * n * C);
    double *A = malloc(sizeof(double) * n * C * nlm);
    double *q = malloc(sizeof(double) * n * 2 * C);
    double *h = malloc(sizeof(double) * n * C);
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < C; ++c) s0[(long)i * C + c] = m.emb[species[i] * C + c];
    mp_layer_forward(&m, 0, n, &E, s0, A, q, h, s1);

    double *V = malloc(sizeof(double) * n * nl * 3);
    double *Q = malloc(sizeof(double) * n * H * nc);
    double *Kk = malloc(sizeof(double) * n * H * nc);
    for (int i = 0; i < n; ++i) {
        for (int hh = 0; hh < nl; ++hh)
            for (int a = 0; a < 3; ++a) {
                double acc = 0.0;
                for (int c = 0; c < C; ++c) acc += m.U[hh * C + c] * A[((long)i * C + c) * nlm + 1 + a];
                V[((long)i * nl + hh) * 3 + a] = acc;
            }
        for (int hh = 0; hh < H; ++hh)
            for (int k = 0; k < nc; ++k) {
                double aq = 0.0, ak = 0.0;
                for (int c = 0; c < C; ++c) {
                    aq += m.Wq[(hh * nc + k) * C + c] * s1[(long)i * C + c];
                    ak += m.Wk[(hh * nc + k) * C + c] * s1[(long)i * C + c];
                }
                Q[((long)i * H + hh) * nc + k] = aq;
                Kk[((long)i * H + hh) * nc + k] = ak;
            }
    }

    /* rows of the (symmetric) neighbour list: edges are grouped by i */
    for (int i = 0; i < 3 * n; ++i) F[i] = 0.0;
    double inv_sqrt_nc = 1.0 / sqrt((double)nc);
    for (long e = 0; e < E.n; ++e) {
        int i = E.i[e], j = E.j[e];
        double r = E.r[e];
        double fc = orc_envelope(r / m.rc, m.p);
        double B[64];
        for (int hh = 0; hh < K; ++hh) B[hh] = orc_bessel(hh + 1, r, m.rc);
        double Fij[3], Fji[3];
        for (int dir = 0; dir < 2; ++dir) {
            /* dir 0: F_ij (receiver i, vector R_ij/r); dir 1: F_ji (R_ji/r = -R_ij/r) */
            int a_ = dir == 0 ? i : j, b_ = dir == 0 ? j : i;
            double sgn = dir == 0 ? 1.0 : -1.0;
            double cc[64];
            for (int hh = 0; hh < H; ++hh) {
                double acc = 0.0;
                for (int k = 0; k < nc; ++k)
                    acc += Q[((long)a_ * H + hh) * nc + k] * Kk[((long)b_ * H + hh) * nc + k];
                cc[hh] = inv_sqrt_nc * acc;
            }
            double S = 0.0;
            for (int hh = 0; hh < K; ++hh) S += cc[hh] * B[hh];
            double vec[3];
            for (int a = 0; a < 3; ++a) {
                vec[a] = sgn * E.d[3 * e + a] / r;
                for (int hh = 0; hh < nl; ++hh) vec[a] += cc[K + hh] * V[((long)a_ * nl + hh) * 3 + a];
            }
            double *out = dir == 0 ? Fij : Fji;
            for (int a = 0; a < 3; ++a) out[a] = S * vec[a] * fc;
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] += m.scale * (Fij[a] - Fji[a]);
        for (int a = 0; a < 3; ++a) W += m.scale * Fij[a] * E.d[3 * e + a];
    }
    if (fast_terms) {
        double *Fb = malloc(sizeof(double) * 3 * n), Wb = 0.0;
        orc_prior(n, x, species, NULL, box, n_bonds, bonds, bond_r0, pr, fast_terms, Fb, &Wb);
        for (int i = 0; i < 3 * n; ++i) F[i] += Fb[i];
        W += Wb;
        free(Fb);
    }
    if (virial) *virial = W;
    double net[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) net[a] += F[3 * i + a];
    if (net_pre) for (int a = 0; a < 3; ++a) net_pre[a] = net[a];
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) F[3 * i + a] -= net[a] / n;
    free(s0); free(s1); free(A); free(q); free(h); free(V); free(Q); free(Kk);
    edges_free(&E);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Gaussian draws      */
/* ------------------------------------------------------------------------ */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Ten rounds; between rounds the key is bumped by the Weyl constants. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c[0], &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Raw words for (seed, replica, step, atom): key = (seed_lo, seed_hi),
 * counter = (atom, replica, step_lo, step_hi). */
void orc_noise_words(uint64_t seed, uint32_t replica, uint64_t step, uint32_t atom, uint32_t w[4])
{
    uint32_t ctr[4] = {atom, replica, (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

/* Box-Muller on (w0, w1) -> (g0, g1) and on (w2, w3) -> g2; u = (w + 1/2) 2^-32. */
void orc_gauss3(uint64_t seed, uint32_t replica, uint64_t step, uint32_t atom, double g[3])
{
    uint32_t w[4];
    orc_noise_words(seed, replica, step, atom, w);
    double u[4];
    for (int k = 0; k < 4; ++k) u[k] = ((double)w[k] + 0.5) * (1.0 / 4294967296.0);
    double r01 = sqrt(-2.0 * log(u[0])), r23 = sqrt(-2.0 * log(u[2]));
    g[0] = r01 * cos(2.0 * M_PI * u[1]);
    g[1] = r01 * sin(2.0 * M_PI * u[1]);
    g[2] = r23 * cos(2.0 * M_PI * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Masses and friction                                                       */
/* ------------------------------------------------------------------------ */

/* Hydrogen mass repartitioning: every H gains delta_h; the molecule's total
 * gain is removed from its heavy atoms in proportion to their masses, so each
 * molecule keeps its mass. Molecules without heavy atoms are unchanged. */
void orc_hmr_masses(int n, const uint8_t *species, const int *mol_id, const double *m_in,
                    double delta_h, double *m_out)
{
    int max_mol = 0;
    for (int i = 0; i < n; ++i) if (mol_id[i] > max_mol) max_mol = mol_id[i];
    double *gain = calloc(max_mol + 1, sizeof(double));
    double *heavy = calloc(max_mol + 1, sizeof(double));
    for (int i = 0; i < n; ++i) {
        if (species[i] == ORC_SP_H) gain[mol_id[i]] += delta_h;
        else heavy[mol_id[i]] += m_in[i];
    }
    for (int i = 0; i < n; ++i) {
        int mo = mol_id[i];
        if (heavy[mo] == 0.0) { m_out[i] = m_in[i]; continue; }
        if (species[i] == ORC_SP_H) m_out[i] = m_in[i] + delta_h;
        else m_out[i] = m_in[i] - gain[mo] * m_in[i] / heavy[mo];
    }
    free(gain); free(heavy);
}

/* O-step constants per species: c1 = exp(-gamma dt), c2 = sqrt((1-c1^2) kB T),
 * with gamma in 1/ps and kB T converted to A^2/fs^2 * amu. */
void orc_gamma_table(int n_species, const double *gamma_ps, double dt_fs, double T,
                     double *c1, double *c2)
{
    for (int s = 0; s < n_species; ++s) {
        c1[s] = exp(-gamma_ps[s] * 1e-3 * dt_fs);
        c2[s] = sqrt((1.0 - c1[s] * c1[s]) * ORC_KB * T * ORC_ACC_CONV);
    }
}

/* ------------------------------------------------------------------------ */
/* Integrators                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    const uint8_t *species;
    const int *mol_id;
    const double *box;
    int n_bonds;
    const int *bonds;
    const double *bond_r0;
    const double *prior;     /* [k_bond, eps, sigma, lj_rc, lj_p] */
    const int *cmi; const double *cmr; const double *cblob;     /* conservative */
    const int *nmi; const double *nmr; const double *nblob;     /* NC */
    const double *mass;      /* simulation masses */
    const double *gamma_ps;  /* per species */
    double T;
    uint64_t seed;
    uint32_t replica;
    int inner_mode;          /* 0: NC + bonds + F_rep, 1: full -grad U, 2: bonds only */
    int outer_mode;          /* 0: -grad(U_MP + bonds + LJ + E_rep), 1: bonds only */
    int thermostat;          /* 0: Langevin O-step, 1: Fast Forward Langevin */
} md_t;

/* Slow force F_full = -grad U (U = U_MP + bonds + LJ) or a reduced U. */
static double full_force(const md_t *md, const double *x, double *F)
{
    double *Fp = malloc(sizeof(double) * 3 * md->n);
    double E = 0.0;
    if (md->outer_mode == 0) {
        E = orc_cons_energy_forces(md->n, x, md->species, md->box, md->cmi, md->cmr, md->cblob, F);
        E += orc_prior(md->n, x, md->species, md->mol_id, md->box, md->n_bonds, md->bonds,
                       md->bond_r0, md->prior, 7, Fp, NULL);
    } else {
        for (int i = 0; i < 3 * md->n; ++i) F[i] = 0.0;
        E = orc_prior(md->n, x, md->species, md->mol_id, md->box, md->n_bonds, md->bonds,
                      md->bond_r0, md->prior, 1, Fp, NULL);
    }
    for (int i = 0; i < 3 * md->n; ++i) F[i] += Fp[i];
    free(Fp);
    return E;
}

/* Fast (inner) force F_S; returns its virial proxy (pair form; 0 for the
 * full force, which has no pair form). */
static double inner_force(const md_t *md, const double *x, double *F)
{
    double W = 0.0;
    if (md->inner_mode == 0) {
        orc_nc_forces(md->n, x, md->species, md->box, md->nmi, md->nmr, md->nblob, md->n_bonds,
                      md->bonds, md->bond_r0, md->prior, 5, F, NULL, &W);
    } else if (md->inner_mode == 1) {
        full_force(md, x, F);
    } else {
        orc_prior(md->n, x, md->species, md->mol_id, md->box, md->n_bonds, md->bonds, md->bond_r0,
                  md->prior, 1, F, &W);
    }
    return W;
}

static void kick(int n, double *v, const double *F, const double *F2, double h, const double *mass)
{
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double f = F[3 * i + a] - (F2 ? F2[3 * i + a] : 0.0);
            v[3 * i + a] += h * ORC_ACC_CONV * f / mass[i];
        }
}

static void drift(int n, double *x, const double *v, double h)
{
    for (int i = 0; i < 3 * n; ++i) x[i] += h * v[i];
}

/* O-step: w_i = c1 v_i + c2 sqrt(1/m_i) G_i, G from Philox at (seed, replica,
 * step, i). Langevin: v_i <- w_i. Fast Forward Langevin (Sec. 2, "High
 * Hydrogen Friction", the FFL update): v_i <- |w_i| v_i / |v_i|, the norm
 * taken of each atom's 3-vector; an atom at rest takes w_i. */
static void ostep(const md_t *md, double *v, double dt, uint64_t step)
{
    double c1[16], c2[16];
    orc_gamma_table(5, md->gamma_ps, dt, md->T, c1, c2);
    for (int i = 0; i < md->n; ++i) {
        double g[3], w[3];
        orc_gauss3(md->seed, md->replica, step, (uint32_t)i, g);
        int s = md->species[i];
        for (int a = 0; a < 3; ++a)
            w[a] = c1[s] * v[3 * i + a] + c2[s] * sqrt(1.0 / md->mass[i]) * g[a];
        double nv = 0.0, nw = 0.0;
        for (int a = 0; a < 3; ++a) {
            nv += v[3 * i + a] * v[3 * i + a];
            nw += w[a] * w[a];
        }
        if (md->thermostat == 1 && nv > 0.0) {
            double f = sqrt(nw) / sqrt(nv);
            for (int a = 0; a < 3; ++a) v[3 * i + a] *= f;
        } else {
            for (int a = 0; a < 3; ++a) v[3 * i + a] = w[a];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Barostat                                                                  */
/* ------------------------------------------------------------------------ */
/* Reading of Sec. 3's "Bussi's barostat" (stochastic, isotropic): the volume
 * follows epsilon = ln(V)/3 with a piston momentum p_eps (kcal/mol fs) of mass
 * W = (N_f + 3) kB T tau_P^2, friction 1/tau_P and matching noise (a Langevin
 * piston); the particles couple to it as in the isotropic Martyna-Tobias-Klein
 * equations: dx/dt = v + (p_eps/W) x, dv/dt = ... - (1 + 3/N_f)(p_eps/W) v,
 * dp_eps/dt = (1 + 3/N_f) 2K - Wvir - 3 V P_ext, with Wvir = -sum_i F_i . q_i
 * the virial estimator of Sec. 2 (the pair form). Per outer step Delta:
 * p_eps += Delta/2 G; p_eps <- c p_eps + sqrt((1 - c^2) W kB T) xi
 * (c = exp(-Delta/tau_P), xi from Philox at (seed, replica, step, 2^32 - 1));
 * the outer step with p_eps fixed, each A half-step of length h being
 * x <- x e^(b h) + h phi(b h) v, v <- v e^(-a h), box <- box e^(b h)
 * (b = p_eps/W, a = (1 + 3/N_f) b, phi(z) = (e^z - 1)/z: the exact flow of
 * dx/dt = v + b x for constant v); then G <- its value at the step's end and
 * p_eps += Delta/2 G. N_f = 3 n. */
#define ORC_KCAL_PER_A3_PER_ATM (101325.0 * 6.02214076e23 * 1e-30 / 4184.0)

double orc_baro_mass(int n, double T, double tau_p_fs)
{
    return (3.0 * n + 3.0) * ORC_KB * T * tau_p_fs * tau_p_fs;
}

/* Generalised force on the piston: (1 + 3/N_f) 2K - Wvir - 3 V P_ext. */
double orc_baro_force(int n, double K, double wvir, const double *box, double p_atm)
{
    double V = box[0] * box[1] * box[2];
    return (1.0 + 3.0 / (3.0 * n)) * 2.0 * K - wvir - 3.0 * V * p_atm * ORC_KCAL_PER_A3_PER_ATM;
}

/* Kinetic energy sum_i m_i v_i^2 / 2 in kcal/mol. */
double orc_kinetic(int n, const double *v, const double *mass)
{
    double K = 0.0;
    for (int i = 0; i < n; ++i)
        K += 0.5 * mass[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    return K / ORC_ACC_CONV;
}

/* A half-step with the piston: the exact flow of dx/dt = v + b x (v fixed),
 * then v <- v e^(-a h), box <- box e^(b h). */
void orc_baro_drift(int n, double *x, double *v, double *box, double h, double b, double a)
{
    double z = b * h, e = exp(z), phi = z != 0.0 ? expm1(z) / z : 1.0, s = exp(-a * h);
    for (int i = 0; i < 3 * n; ++i) {
        x[i] = x[i] * e + h * phi * v[i];
        v[i] *= s;
    }
    for (int k = 0; k < 3; ++k) box[k] *= e;
}

/* Virial of the full force, dU(lambda q, lambda L)/dlambda at 1, by central
 * differences (the pair form's definition; -sum_i F_i . q_i in open space). */
static double full_virial_fd(const md_t *md, const double *x)
{
    const double h = 1e-6;
    int n = md->n;
    double *xs = malloc(sizeof(double) * 3 * n), *F = malloc(sizeof(double) * 3 * n), bs[3], U[2];
    md_t m2 = *md;
    m2.box = bs;
    for (int sgn = 0; sgn < 2; ++sgn) {
        double lam = sgn ? 1.0 - h : 1.0 + h;
        for (int i = 0; i < 3 * n; ++i) xs[i] = x[i] * lam;
        for (int k = 0; k < 3; ++k) bs[k] = md->box[k] * lam;
        U[sgn] = full_force(&m2, xs, F);
    }
    free(xs); free(F);
    return (U[0] - U[1]) / (2.0 * h);
}

/* Algorithm 1 (DMTS-NC integration step), repeated n_outer times.
 * state: x, v, F (full force -grad U), F_nc (fast force), *step (global inner
 * step index, advanced by n per outer step), *first (force cache flag).
 * virial_avg (nullable): average over the n inner force evaluations of the
 * last outer step of the fast force's virial proxy (Sec. 2 "Computation of
 * the virial term in NPT").
 * ints: [n_atoms, n_bonds, inner_mode, outer_mode, n_inner, replica, thermostat]
 * reals: [dt_outer, T]
 * Returns the last evaluated potential energy U. */
double orc_respa_run(const int *ints, const double *reals, uint64_t seed,
                     const uint8_t *species, const int *mol_id, const double *box,
                     const int *bonds, const double *bond_r0, const double *prior,
                     const int *cmi, const double *cmr, const double *cblob,
                     const int *nmi, const double *nmr, const double *nblob,
                     const double *mass, const double *gamma_ps,
                     int n_outer, double *x, double *v, double *F, double *F_nc,
                     uint64_t *step, int *first, double *virial_avg,
                     const double *baro_par, double *box_io, double *baro)
{
    md_t md = {ints[0], species, mol_id, box, ints[1], bonds, bond_r0, prior,
               cmi, cmr, cblob, nmi, nmr, nblob, mass, gamma_ps, reals[1], seed,
               (uint32_t)ints[5], ints[2], ints[3], ints[6]};
    int n = md.n, n_in = ints[4];
    double Delta = reals[0], delta = Delta / n_in, U = 0.0;
    /* barostat (nullable): baro_par = [P_ext atm, tau_P ps], box_io the box it
     * moves, baro = [p_eps, G, have_G] */
    const int npt = baro_par && box_io && baro && box_io[0] > 0.0;
    double Wp = 0.0, cP = 0.0, b = 0.0, a = 0.0;
    if (npt) {
        md.box = box_io;
        Wp = orc_baro_mass(n, md.T, baro_par[1] * 1e3);
        cP = exp(-Delta / (baro_par[1] * 1e3));
    }
    if (*first) {
        inner_force(&md, x, F_nc);
        U = full_force(&md, x, F);
        *first = 0;
    }
    for (int o = 0; o < n_outer; ++o) {
        double wsum = 0.0, wlast = 0.0;
        if (npt) {
            if (baro[2] == 0.0) {     /* no estimator yet: the full force's virial */
                baro[1] = orc_baro_force(n, orc_kinetic(n, v, mass), full_virial_fd(&md, x), box_io, baro_par[0]);
                baro[2] = 1.0;
            }
            double g[3];
            orc_gauss3(md.seed, md.replica, *step, 0xFFFFFFFFu, g);
            baro[0] += 0.5 * Delta * baro[1];
            baro[0] = cP * baro[0] + sqrt((1.0 - cP * cP) * Wp * ORC_KB * md.T) * g[0];
            b = baro[0] / Wp;
            a = (1.0 + 3.0 / (3.0 * n)) * b;
        }
        kick(n, v, F, F_nc, Delta / 2.0, mass);                /* v += D/2 M^-1 (F - F_NC) */
        for (int k = 0; k < n_in; ++k) {
            kick(n, v, F_nc, NULL, delta / 2.0, mass);          /* B */
            if (npt) orc_baro_drift(n, x, v, box_io, delta / 2.0, b, a);
            else drift(n, x, v, delta / 2.0);                   /* A */
            ostep(&md, v, delta, *step);                        /* O, Thermostat(v, D/n) */
            if (npt) orc_baro_drift(n, x, v, box_io, delta / 2.0, b, a);
            else drift(n, x, v, delta / 2.0);                   /* A */
            wlast = inner_force(&md, x, F_nc);                  /* F_NC <- NC(x) */
            wsum += wlast;
            kick(n, v, F_nc, NULL, delta / 2.0, mass);          /* B */
            *step += 1;
        }
        U = full_force(&md, x, F);                              /* F <- large(x) */
        kick(n, v, F, F_nc, Delta / 2.0, mass);                 /* v += D/2 M^-1 (F - F_NC) */
        if (virial_avg) *virial_avg = wsum / n_in;
        if (npt) {
            /* the estimator of Sec. 2 at the step's end: the full force's
             * virial with the fast force's share replaced by its average */
            double west = full_virial_fd(&md, x) - wlast + wsum / n_in;
            baro[1] = orc_baro_force(n, orc_kinetic(n, v, mass), west, box_io, baro_par[0]);
            baro[0] += 0.5 * Delta * baro[1];
        }
    }
    return U;
}

/* Single-time-step BAOAB with the full force, n_steps steps of dt.
 * ints: [n_atoms, n_bonds, outer_mode, replica, thermostat]; reals: [dt, T]. */
double orc_sts_run(const int *ints, const double *reals, uint64_t seed,
                   const uint8_t *species, const int *mol_id, const double *box,
                   const int *bonds, const double *bond_r0, const double *prior,
                   const int *cmi, const double *cmr, const double *cblob,
                   const double *mass, const double *gamma_ps,
                   int n_steps, double *x, double *v, double *F, uint64_t *step, int *first)
{
    md_t md = {ints[0], species, mol_id, box, ints[1], bonds, bond_r0, prior,
               cmi, cmr, cblob, NULL, NULL, NULL, mass, gamma_ps, reals[1], seed,
               (uint32_t)ints[3], 0, ints[2], ints[4]};
    int n = md.n;
    double dt = reals[0], U = 0.0;
    if (*first) {
        U = full_force(&md, x, F);
        *first = 0;
    }
    for (int s = 0; s < n_steps; ++s) {
        kick(n, v, F, NULL, dt / 2.0, mass);
        drift(n, x, v, dt / 2.0);
        ostep(&md, v, dt, *step);
        drift(n, x, v, dt / 2.0);
        U = full_force(&md, x, F);
        kick(n, v, F, NULL, dt / 2.0, mass);
        *step += 1;
    }
    return U;
}
