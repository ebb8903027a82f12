/*
 * Flip Monte Carlo oracle: a plain, slow, FP64 host implementation of the
 * Markov chain of "Molecular motion at the experimental glass transition"
 * (Simon, Barrat, Berthier; arXiv 2506.21290), Sec. II.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA path: every formula
 * below is written out here from the paper and from the schedule definition
 * of the library's interface (the checkerboard reading of the paper's
 * "randomly select a molecule", which the paper leaves open).
 *
 * Build with floating-point contraction disabled (-ffp-contract=off) and
 * without -ffast-math: every FP64 expression is evaluated as written, one
 * IEEE rounding per operation, which is what makes bit-for-bit trajectory
 * comparisons with the GPU's FP64 mode meaningful.
 *
 * Model (Sec. II.A):
 *   - M molecules, 3 atoms each; site i belongs to molecule i/3.  Types
 *     0=A, 1=B, 2=C with diameters sigma_A=0.9, sigma_B=1, sigma_C=1.1.
 *   - WCA on every pair, intra- and intermolecular (Eq. 1):
 *       U = 4 eps ((s/r)^12 - (s/r)^6 + 1/4)  for r < 2^(1/6) s, else 0,
 *     with s = (sigma_a + sigma_b)/2.
 *   - FENE on the three bonds of each triangle (Eq. 2):
 *       U = -33.75 eps ln(1 - (r / (1.5 s))^2).
 *   - Periodic cubic box of side L; number density 3M/L^3 (1.2 in the paper).
 * Moves (Sec. II.B): local atom translations and flips (a flip swaps the types
 * of the two atoms that are not on the chosen median axis), Metropolis
 * acceptance, one MC time step = N = 3M attempts.  Rigid molecule translations
 * and rotations are two further symmetric moves the library offers.
 *
 * Precision-sensitive definitions (shared by specification, not by code, with
 * the GPU FP64 mode):
 *   - positions are 32-bit fixed point per axis, x = q L / 2^32; pair vectors
 *     are the int32 difference of two q's (the minimum image), times h=L/2^32;
 *   - r2 = (dx*dx + dy*dy) + dz*dz;
 *   - WCA: t = s2/r2; s6 = (t*t)*t; U = e4*((s6*s6) - s6) + eps, zero unless
 *     r2 < rc2, rc2 = C13 * s2 with C13 the double nearest 2^(1/3);
 *   - FENE: U = nke * ln(1 - r2/R2), nke = -(K eps), R2 = (R0 s)^2;
 *   - ln is the atanh-series logarithm orc_ln() below (not libm's);
 *   - Delta E of a move = sequential FP64 sum, starting from 0.0, of the terms
 *     (phi_new - phi_old), ordered by moved site (ascending index) and then by
 *     partner index (ascending); rotations append the three intramolecular
 *     pairs (s0,s1), (s0,s2), (s1,s2);
 *   - accept iff dE <= 0 or dE <= -(T * ln(u)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { MV_ATOM = 0, MV_FLIP = 1, MV_MOLT = 2, MV_MOLR = 3 };
enum { ST_EVAL = 0, ST_LEFT_CELL = 1, ST_BOND_BREAK = 2, ST_NOT_IN_CELL = 3 };

/* One record per attempted move; the same layout the library's attempt log
 * uses (site, move type, status, accepted flag, Delta E, conditioning scale). */
typedef struct {
    int32_t site, move, status, accepted;
    double dE, scale;
} orc_log_entry;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies; the key */
/* is bumped by the Weyl constants before every round but the first.         */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_at(uint32_t w0, uint32_t w1, uint64_t sweep, uint64_t seed, uint32_t out[4])
{
    uint32_t ctr[4] = { w0, w1, (uint32_t)sweep, (uint32_t)(sweep >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm by argument reduction and the atanh series:             */
/*   x = m 2^e, m in [sqrt(1/2), sqrt(2)],  z = (m-1)/(m+1),                 */
/*   ln x = e ln2 + 2 (z + z^3/3 + z^5/5 + ...),                             */
/* with |z| <= 0.1716, so twelve terms reach double precision.               */
/* ------------------------------------------------------------------------ */
double orc_ln(double x)
{
    if (x != x) return x;
    if (x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (x == INFINITY) return x;
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0) {                      /* subnormal: scale into the normal range */
        x = x * 0x1p64;
        memcpy(&bits, &x, sizeof bits);
        e = (int)((bits >> 52) & 0x7FF) - 64;
    }
    e -= 1023;
    uint64_t mbits = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double m;
    memcpy(&m, &mbits, sizeof m);      /* m in [1, 2) */
    if (m > 0x1.6a09e667f3bcdp+0) {    /* fold (sqrt2, 2) onto (sqrt(1/2), 1) */
        m = m * 0.5;
        e = e + 1;
    }
    double z = (m - 1.0) / (m + 1.0);
    double w = z * z;
    /* coefficients 2/(2k+1), k = 11 down to 0, Horner in w */
    double s = 2.0 / 23.0;
    s = s * w + 2.0 / 21.0;
    s = s * w + 2.0 / 19.0;
    s = s * w + 2.0 / 17.0;
    s = s * w + 2.0 / 15.0;
    s = s * w + 2.0 / 13.0;
    s = s * w + 2.0 / 11.0;
    s = s * w + 2.0 / 9.0;
    s = s * w + 2.0 / 7.0;
    s = s * w + 2.0 / 5.0;
    s = s * w + 2.0 / 3.0;
    s = s * w + 2.0;
    double series = z * s;
    double el = (double)e * 0x1.62e42fefa39efp-1;   /* double nearest ln 2 */
    return el + series;
}

/* ------------------------------------------------------------------------ */
/* Pair potentials, Eq. (1) and Eq. (2)                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double s2[3][3];    /* sigma_ab^2                          */
    double rc2[3][3];   /* WCA cutoff^2 = 2^(1/3) sigma_ab^2   */
    double R2[3][3];    /* FENE divergence^2 = (R0 sigma_ab)^2 */
    double eps, e4, nke, ke;
} model;

/* pot = {sigma_A, sigma_B, sigma_C, eps, fene_K, fene_R0} */
static void model_init(model *md, const double *pot)
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = (pot[a] + pot[b]) * 0.5;
            double s2 = s * s;
            double R = pot[5] * s;
            md->s2[a][b] = s2;
            md->rc2[a][b] = 0x1.428a2f98d728bp+0 * s2;
            md->R2[a][b] = R * R;
        }
    md->eps = pot[3];
    md->e4 = 4.0 * pot[3];
    md->ke = pot[4] * pot[3];
    md->nke = -md->ke;
}

static double wca(const model *md, double r2, int a, int b)
{
    if (!(r2 < md->rc2[a][b])) return 0.0;
    double t = md->s2[a][b] / r2;
    double s6 = (t * t) * t;
    return md->e4 * ((s6 * s6) - s6) + md->eps;
}

static double fene(const model *md, double r2, int a, int b)
{
    double x = r2 / md->R2[a][b];
    return md->nke * orc_ln(1.0 - x);
}

/* total pair energy of (a,b) at squared distance r2; bonded = same molecule */
static double phi(const model *md, double r2, int a, int b, int bonded)
{
    double u = wca(md, r2, a, b);
    if (bonded) u = u + fene(md, r2, a, b);
    return u;
}

/* Conditioning scale of one pair evaluation: the sum of the magnitudes of the
 * pieces an FP32 evaluation adds up (4eps s^12, 4eps s^6, eps) plus, for a
 * bond, K eps (|ln(1-x)| + x/(1-x)).  Used only to scale tolerances. */
static double mag(const model *md, double r2, int a, int b, int bonded)
{
    double m = 0.0;
    if (r2 < md->rc2[a][b]) {
        double t = md->s2[a][b] / r2;
        double s6 = (t * t) * t;
        m = md->e4 * s6 * s6 + md->e4 * s6 + md->eps;
    }
    if (bonded) {
        double x = r2 / md->R2[a][b];
        m += md->ke * (fabs(log(1.0 - x)) + x / (1.0 - x));
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* Fixed-point geometry                                                      */
/* ------------------------------------------------------------------------ */
static double r2_of(const uint32_t *a, const uint32_t *b, double h)
{
    int32_t d0 = (int32_t)(b[0] - a[0]);
    int32_t d1 = (int32_t)(b[1] - a[1]);
    int32_t d2 = (int32_t)(b[2] - a[2]);
    double dx = (double)d0 * h, dy = (double)d1 * h, dz = (double)d2 * h;
    return (dx * dx + dy * dy) + dz * dz;
}

/* Wrap x into [0, L) and quantise to 32 bits: q = floor(frac(x/L) 2^32). */
uint32_t orc_quantize(double x, double L)
{
    double t = x / L;
    t = t - floor(t);
    double v = floor(t * 4294967296.0);
    if (v >= 4294967296.0) v = 0.0;
    return (uint32_t)v;
}

void orc_quantize_all(int n, const double *x, double L, uint32_t *q)
{
    for (int i = 0; i < n; ++i) q[i] = orc_quantize(x[i], L);
}

static uint32_t cell_axis(uint32_t qv, uint32_t shift, int nc)
{
    return (uint32_t)(((uint64_t)(uint32_t)(qv + shift) * (uint64_t)nc) >> 32);
}

static int cell_of(const uint32_t *q, const uint32_t *shift, int nc)
{
    int cx = (int)cell_axis(q[0], shift[0], nc);
    int cy = (int)cell_axis(q[1], shift[1], nc);
    int cz = (int)cell_axis(q[2], shift[2], nc);
    return (cz * nc + cy) * nc + cx;
}

static int colour_of_cell(int c, int nc)
{
    int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    return (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
}

/* displacement half-width in fixed-point units: floor(d / L * 2^32) */
static int64_t half_width(double d, double L)
{
    return (int64_t)floor(d / L * 4294967296.0);
}

/* uniform integer in [-D, D] from one 32-bit word */
static int32_t uniform_disp(uint32_t w, int64_t D)
{
    uint64_t span = (uint64_t)(2 * D + 1);
    return (int32_t)((int64_t)(((uint64_t)w * span) >> 32) - D);
}

/* Move-type thresholds on a 32-bit word from the cumulative probabilities;
 * a threshold past which only zero-probability types remain is 2^32. */
static void move_thresholds(const double *p, uint64_t thr[3])
{
    double c = 0.0;
    for (int k = 0; k < 3; ++k) {
        c = c + p[k];
        int tail_zero = 1;
        for (int m = k + 1; m < 4; ++m)
            if (p[m] != 0.0) tail_zero = 0;
        double v = floor(c * 4294967296.0);
        if (tail_zero || v >= 4294967296.0) thr[k] = 4294967296ull;
        else thr[k] = (uint64_t)v;
    }
}

static int move_type(uint32_t w, const uint64_t thr[3])
{
    if ((uint64_t)w < thr[0]) return MV_ATOM;
    if ((uint64_t)w < thr[1]) return MV_FLIP;
    if ((uint64_t)w < thr[2]) return MV_MOLT;
    return MV_MOLR;
}

/* ------------------------------------------------------------------------ */
/* Total energy by brute force over all pairs i < j (minimum image)         */
/* ------------------------------------------------------------------------ */
double orc_energy(double L, int M, const uint32_t *q, const int32_t *t, const double *pot)
{
    model md;
    model_init(&md, pot);
    double h = L / 4294967296.0;
    int N = 3 * M;
    double E = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double r2 = r2_of(q + 3 * i, q + 3 * j, h);
            E = E + phi(&md, r2, t[i], t[j], (i / 3) == (j / 3));
        }
    return E;
}

/* Energy of one site against all others (used by tests as an independent
 * route to Delta E). */
double orc_site_energy(double L, int M, const uint32_t *q, const int32_t *t, const double *pot, int i)
{
    model md;
    model_init(&md, pot);
    double h = L / 4294967296.0;
    double E = 0.0;
    for (int j = 0; j < 3 * M; ++j) {
        if (j == i) continue;
        E = E + phi(&md, r2_of(q + 3 * i, q + 3 * j, h), t[i], t[j], (i / 3) == (j / 3));
    }
    return E;
}

/* ------------------------------------------------------------------------ */
/* The chain                                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    double L, h, inv_h, T;
    int M, N, nc;
    uint32_t *q;        /* 3N, site-major */
    int64_t *X;         /* 3N, unwrapped fixed point */
    int32_t *t;         /* N */
    model md;
    uint64_t thr[3];
    int64_t D_atom, D_mol;
    double rot_a;
    uint32_t shift[3];
} chain;

/* Sum of (phi_new - phi_old) for moved site s (old position qo, new position
 * qn, old type to, new type tn) against every site j not in the moved set
 * `moved` (n_moved entries), ascending j.  Adds to *dE and *scale. */
static void site_terms(const chain *c, int s, const uint32_t *qo, const uint32_t *qn, int to, int tn,
                       const int *moved, int n_moved, double *dE, double *scale)
{
    int m = s / 3;
    for (int j = 0; j < c->N; ++j) {
        int skip = 0;
        for (int k = 0; k < n_moved; ++k)
            if (moved[k] == j) skip = 1;
        if (skip) continue;
        int bonded = (j / 3) == m;
        int tj = c->t[j];
        double r2o = r2_of(qo, c->q + 3 * j, c->h);
        double r2n = (qn == qo) ? r2o : r2_of(qn, c->q + 3 * j, c->h);
        double un = phi(&c->md, r2n, tn, tj, bonded);
        double uo = phi(&c->md, r2o, to, tj, bonded);
        *dE = *dE + (un - uo);
        *scale = *scale + mag(&c->md, r2n, tn, tj, bonded) + mag(&c->md, r2o, to, tj, bonded);
    }
}

static int in_cell(const chain *c, const uint32_t *qv, int cell)
{
    return cell_of(qv, c->shift, c->nc) == cell;
}

/* One attempted move.  Returns accepted flag; fills the log entry. */
static int attempt(chain *c, int cell, const int *members, int n, int a, uint64_t sweep,
                   uint64_t seed, double *e_run, uint64_t *counters, orc_log_entry *lg)
{
    uint32_t b0[4], b1[4];
    philox_at((uint32_t)(2 * a), (uint32_t)cell, sweep, seed, b0);
    philox_at((uint32_t)(2 * a + 1), (uint32_t)cell, sweep, seed, b1);
    int i = members[(int)(((uint64_t)b0[0] * (uint64_t)n) >> 32)];
    int mv = move_type(b0[1], c->thr);
    uint64_t u52 = ((uint64_t)b0[2] << 20) | (uint64_t)(b0[3] >> 12);
    double u = (double)(2 * u52 + 1) * 0x1p-53;
    int m = i / 3;
    int status = ST_EVAL;
    double dE = 0.0, scale = 0.0;
    uint32_t qn[3][3];          /* proposed positions of up to three sites */
    int moved[3];
    int n_moved = 0;
    int flip_p = -1, flip_q = -1;

    counters[mv] += 1;

    if (mv == MV_ATOM) {
        int64_t D = c->D_atom;
        for (int k = 0; k < 3; ++k)
            qn[0][k] = c->q[3 * i + k] + (uint32_t)uniform_disp(b1[k], D);
        moved[0] = i;
        n_moved = 1;
        if (!in_cell(c, qn[0], cell)) status = ST_LEFT_CELL;
        if (status == ST_EVAL)
            for (int j = 3 * m; j < 3 * m + 3; ++j) {
                if (j == i) continue;
                if (!(r2_of(qn[0], c->q + 3 * j, c->h) < c->md.R2[c->t[i]][c->t[j]])) status = ST_BOND_BREAK;
            }
        if (status == ST_EVAL)
            site_terms(c, i, c->q + 3 * i, qn[0], c->t[i], c->t[i], moved, 1, &dE, &scale);
    } else if (mv == MV_FLIP) {
        int axis = (int)(((uint64_t)b1[3] * 3u) >> 32);
        int sa = 3 * m + axis;
        int others[2], k2 = 0;
        for (int j = 3 * m; j < 3 * m + 3; ++j)
            if (j != sa) others[k2++] = j;
        flip_p = others[0];
        flip_q = others[1];
        if (!in_cell(c, c->q + 3 * flip_p, cell) || !in_cell(c, c->q + 3 * flip_q, cell)) status = ST_NOT_IN_CELL;
        int tp = c->t[flip_p], tq = c->t[flip_q], ta = c->t[sa];
        if (status == ST_EVAL) {
            if (!(r2_of(c->q + 3 * flip_p, c->q + 3 * sa, c->h) < c->md.R2[tq][ta])) status = ST_BOND_BREAK;
            if (!(r2_of(c->q + 3 * flip_q, c->q + 3 * sa, c->h) < c->md.R2[tp][ta])) status = ST_BOND_BREAK;
        }
        if (status == ST_EVAL) {
            moved[0] = flip_p;
            moved[1] = flip_q;
            site_terms(c, flip_p, c->q + 3 * flip_p, c->q + 3 * flip_p, tp, tq, moved, 2, &dE, &scale);
            site_terms(c, flip_q, c->q + 3 * flip_q, c->q + 3 * flip_q, tq, tp, moved, 2, &dE, &scale);
        }
    } else {
        for (int k = 0; k < 3; ++k) moved[k] = 3 * m + k;
        n_moved = 3;
        for (int k = 0; k < 3; ++k)
            if (!in_cell(c, c->q + 3 * moved[k], cell)) status = ST_NOT_IN_CELL;
        if (mv == MV_MOLT) {
            int32_t d[3];
            for (int ax = 0; ax < 3; ++ax) d[ax] = uniform_disp(b1[ax], c->D_mol);
            for (int k = 0; k < 3; ++k)
                for (int ax = 0; ax < 3; ++ax) qn[k][ax] = c->q[3 * moved[k] + ax] + (uint32_t)d[ax];
        } else {
            /* rotation about the centroid by the unit quaternion (1, a v)/|.|,
             * v uniform in (-1,1)^3; v -> -v gives the inverse rotation. */
            const uint32_t *q0 = c->q + 3 * moved[0];
            double rel[3][3], cen[3];
            for (int k = 0; k < 3; ++k)
                for (int ax = 0; ax < 3; ++ax)
                    rel[k][ax] = (double)(int32_t)(c->q[3 * moved[k] + ax] - q0[ax]) * c->h;
            for (int ax = 0; ax < 3; ++ax) cen[ax] = ((rel[0][ax] + rel[1][ax]) + rel[2][ax]) / 3.0;
            double vw = 1.0;
            double vx = c->rot_a * (((double)b1[0] + 0.5) * 0x1p-31 - 1.0);
            double vy = c->rot_a * (((double)b1[1] + 0.5) * 0x1p-31 - 1.0);
            double vz = c->rot_a * (((double)b1[2] + 0.5) * 0x1p-31 - 1.0);
            double ww = vw * vw, xx = vx * vx, yy = vy * vy, zz = vz * vz;
            double xy = vx * vy, xz = vx * vz, yz = vy * vz, wx = vw * vx, wy = vw * vy, wz = vw * vz;
            double n2 = ((ww + xx) + yy) + zz;
            double R[3][3];
            R[0][0] = (((ww + xx) - yy) - zz) / n2;
            R[0][1] = (2.0 * (xy - wz)) / n2;
            R[0][2] = (2.0 * (xz + wy)) / n2;
            R[1][0] = (2.0 * (xy + wz)) / n2;
            R[1][1] = (((ww - xx) + yy) - zz) / n2;
            R[1][2] = (2.0 * (yz - wx)) / n2;
            R[2][0] = (2.0 * (xz - wy)) / n2;
            R[2][1] = (2.0 * (yz + wx)) / n2;
            R[2][2] = (((ww - xx) - yy) + zz) / n2;
            for (int k = 0; k < 3; ++k) {
                double p[3];
                for (int ax = 0; ax < 3; ++ax) p[ax] = rel[k][ax] - cen[ax];
                for (int ax = 0; ax < 3; ++ax) {
                    double np = ((R[ax][0] * p[0] + R[ax][1] * p[1]) + R[ax][2] * p[2]) + cen[ax];
                    int64_t nq = (int64_t)floor(np * c->inv_h + 0.5);
                    qn[k][ax] = q0[ax] + (uint32_t)nq;
                }
            }
        }
        if (status == ST_EVAL)
            for (int k = 0; k < 3; ++k)
                if (!in_cell(c, qn[k], cell)) status = ST_LEFT_CELL;
        if (status == ST_EVAL && mv == MV_MOLR)
            for (int k = 0; k < 3; ++k)
                for (int l = k + 1; l < 3; ++l)
                    if (!(r2_of(qn[k], qn[l], c->h) < c->md.R2[c->t[moved[k]]][c->t[moved[l]]])) status = ST_BOND_BREAK;
        if (status == ST_EVAL) {
            for (int k = 0; k < 3; ++k)
                site_terms(c, moved[k], c->q + 3 * moved[k], qn[k], c->t[moved[k]], c->t[moved[k]], moved, 3, &dE, &scale);
            if (mv == MV_MOLR) {
                static const int pk[3] = { 0, 0, 1 }, pl[3] = { 1, 2, 2 };
                for (int pr = 0; pr < 3; ++pr) {
                    int k = pk[pr], l = pl[pr];
                    int tk = c->t[moved[k]], tl = c->t[moved[l]];
                    double r2o = r2_of(c->q + 3 * moved[k], c->q + 3 * moved[l], c->h);
                    double r2n = r2_of(qn[k], qn[l], c->h);
                    dE = dE + (phi(&c->md, r2n, tk, tl, 1) - phi(&c->md, r2o, tk, tl, 1));
                    scale = scale + mag(&c->md, r2n, tk, tl, 1) + mag(&c->md, r2o, tk, tl, 1);
                }
            }
        }
    }

    int accepted = 0;
    if (status == ST_EVAL) {
        if (dE <= 0.0) accepted = 1;
        else {
            double thr = -(c->T * orc_ln(u));
            accepted = dE <= thr;
        }
    }
    if (accepted) {
        if (mv == MV_FLIP) {
            int tmp = c->t[flip_p];
            c->t[flip_p] = c->t[flip_q];
            c->t[flip_q] = tmp;
        } else {
            for (int k = 0; k < n_moved; ++k)
                for (int ax = 0; ax < 3; ++ax) {
                    int s = moved[k];
                    int32_t d = (int32_t)(qn[k][ax] - c->q[3 * s + ax]);
                    c->X[3 * s + ax] += d;
                    c->q[3 * s + ax] = qn[k][ax];
                }
        }
        *e_run = *e_run + dE;
        counters[4 + mv] += 1;
    }
    if (lg) {
        lg->site = i;
        lg->move = mv;
        lg->status = status;
        lg->accepted = accepted;
        lg->dE = status == ST_EVAL ? dE : NAN;
        lg->scale = status == ST_EVAL ? scale : NAN;
    }
    return accepted;
}

/* Cell shift of a sweep: three 32-bit words of the Philox block at counter
 * (0xFFFFFFFF, 0xFFFFFFFF, sweep). */
void orc_sweep_shift(uint64_t sweep, uint64_t seed, uint32_t shift[3])
{
    uint32_t o[4];
    philox_at(0xFFFFFFFFu, 0xFFFFFFFFu, sweep, seed, o);
    shift[0] = o[0]; shift[1] = o[1]; shift[2] = o[2];
}

/*
 * Run n_sweeps sweeps of the checkerboard schedule.
 *   q, X, t  : state (updated in place), site-major, N = 3M sites
 *   pot      : {sigma_A, sigma_B, sigma_C, eps, fene_K, fene_R0}
 *   mix      : {p_atom, p_flip, p_mol_trans, p_mol_rot, d_atom, d_mol, rot_a}
 *   nc       : cells per axis (even, >= 2)
 *   counters : attempts[4] then accepts[4] (accumulated)
 *   log      : NULL or n_sweeps * N entries, entry (s, cell_start[cell] + a)
 * Sweep k: shift from orc_sweep_shift(sweep0+k); for colour 0..7, for each
 * cell of that colour in ascending id, n = occupancy, attempts a = 0..n-1.
 */
int orc_run(double L, int M, uint32_t *q, int64_t *X, int32_t *t, const double *pot, int nc,
            uint64_t seed, uint64_t sweep0, int n_sweeps, double T, const double *mix,
            double *e_run, uint64_t *counters, orc_log_entry *log)
{
    if (nc < 2 || (nc & 1) || M < 1) return -1;
    chain c;
    memset(&c, 0, sizeof c);
    c.L = L;
    c.h = L / 4294967296.0;
    c.inv_h = 4294967296.0 / L;
    c.T = T;
    c.M = M;
    c.N = 3 * M;
    c.nc = nc;
    c.q = q;
    c.X = X;
    c.t = t;
    model_init(&c.md, pot);
    move_thresholds(mix, c.thr);
    c.D_atom = half_width(mix[4], L);
    c.D_mol = half_width(mix[5], L);
    c.rot_a = mix[6];

    int ncell = nc * nc * nc;
    int *cellid = (int *)malloc(sizeof(int) * c.N);
    int *count = (int *)malloc(sizeof(int) * ncell);
    int *start = (int *)malloc(sizeof(int) * (ncell + 1));
    int *fill = (int *)malloc(sizeof(int) * ncell);
    int *members = (int *)malloc(sizeof(int) * c.N);
    if (!cellid || !count || !start || !fill || !members) return -2;

    for (int s = 0; s < n_sweeps; ++s) {
        uint64_t sweep = sweep0 + (uint64_t)s;
        orc_sweep_shift(sweep, seed, c.shift);
        /* stable counting sort of site indices by cell */
        memset(count, 0, sizeof(int) * ncell);
        for (int i = 0; i < c.N; ++i) {
            cellid[i] = cell_of(c.q + 3 * i, c.shift, nc);
            count[cellid[i]] += 1;
        }
        start[0] = 0;
        for (int k = 0; k < ncell; ++k) start[k + 1] = start[k] + count[k];
        memcpy(fill, start, sizeof(int) * ncell);
        for (int i = 0; i < c.N; ++i) members[fill[cellid[i]]++] = i;

        for (int colour = 0; colour < 8; ++colour)
            for (int cell = 0; cell < ncell; ++cell) {
                if (colour_of_cell(cell, nc) != colour) continue;
                int n = count[cell];
                for (int a = 0; a < n; ++a) {
                    orc_log_entry *lg = log ? log + (size_t)s * c.N + start[cell] + a : NULL;
                    attempt(&c, cell, members + start[cell], n, a, sweep, seed, e_run, counters, lg);
                }
            }
    }
    free(cellid); free(count); free(start); free(fill); free(members);
    return 0;
}

/* Pair energy phi(r2) of types (a,b) for tests of the closed forms of Eq. 1-2. */
double orc_phi(double r2, int a, int b, int bonded, const double *pot)
{
    model md;
    model_init(&md, pot);
    return phi(&md, r2, a, b, bonded);
}

/* phi for n squared distances (same types and bond flag), for quadratures in tests. */
void orc_phi_many(int n, const double *r2, int a, int b, int bonded, const double *pot, double *out)
{
    model md;
    model_init(&md, pot);
    for (int i = 0; i < n; ++i) out[i] = phi(&md, r2[i], a, b, bonded);
}

/* Conditioning scale mag(r2) of one pair evaluation of types (a,b), for tests
 * of its closed forms (the FP32 tolerances are measured against it). */
double orc_mag(double r2, int a, int b, int bonded, const double *pot)
{
    model md;
    model_init(&md, pot);
    return mag(&md, r2, a, b, bonded);
}
