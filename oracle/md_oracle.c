/*
 * CPU FP64 oracle for many-body (EAM / second-moment tight-binding) molecular
 * dynamics, after Hou et al., "Molecular dynamics simulations with many-body
 * potentials on multiple GPUs" (arXiv:1212.6332).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA library is checked against. It shares no code, header, table or
 * constant with the CUDA library, and the library never calls it. Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * What it computes, and where the paper defines it:
 *   - per-atom energy E_i = F(rho_i) + 1/2 sum_j V(r_ij)          Eq. (1)
 *   - total energy E_T = sum_i E_i                                Eq. (2)
 *   - force f_i = -sum_j (F'(rho_i)+F'(rho_j)) rho'(r_ij) r_ij/r_ij
 *                 -sum_j V'(r_ij) r_ij/r_ij                        Eq. (3)
 *     with rho_i = sum_{j != i} rho(r_ij)                          (Sec. 2)
 *   - the SETB embedding F = -sqrt(rho)                            (Sec. 4)
 *   - linked-cell neighbour search with 26 neighbouring cells
 *     under periodic boundaries                                    (Sec. 3.2)
 *   - Newton's third law in the CPU pair loops                     (Sec. 4.3)
 *   - Verlet neighbour list with a radius beyond the force cutoff
 *     (a skin)                                                     (Sec. 4.2)
 *   - the electron-phonon friction of the temperature control      Eq. (4)
 *   - the pair virial, the pressure and its Berendsen coupling   Eq. (5)-(6)
 *
 * Two independent routes for Eq. (1)-(3): orc_forces_brute() writes the double
 * sums out over all atom pairs (O(N^2), the definition), and
 * orc_forces_pairs() takes a half list of pairs i<j and applies Newton's third
 * law. The two are compared against each other by the tests.
 *
 * For timing the CPU baseline on all host cores, orc_pairs_cells_par() and
 * orc_forces_pairs_par() split the same loops over OpenMP threads with
 * thread-private sums added in a fixed order (one thread reproduces the
 * serial functions bit for bit); orc_md_run uses them when orc_set_threads()
 * asked for more than one thread. Every pin runs the serial functions.
 *
 * The potential forms (the paper leaves them to the literature):
 *   RGL (Cleri-Rosato) : V(r) = 2A exp(-p(r/r0-1)) S(r),
 *                        rho(r) = xi^2 exp(-2q(r/r0-1)) S(r), F = -sqrt(rho)
 *   Sutton-Chen        : V(r) = eps (a/r)^n S(r), rho(r) = (a/r)^m S(r),
 *                        F = -c eps sqrt(rho)
 *   spline             : V, rho natural cubic splines of knot values on a
 *                        uniform grid over [r_lo, r_hi] (zero for r >= r_hi,
 *                        linear below r_lo); F a natural cubic spline over
 *                        [rho_lo, rho_hi], linear outside.
 *   S(r) is the C2 smoothstep taper 1 - 10x^3 + 15x^4 - 6x^5 with
 *   x = (r - r_taper)/(r_cut - r_taper), S = 1 below r_taper, 0 at r_cut.
 *   F(rho) = F'(rho) = 0 for rho <= 0 (an isolated atom).
 *
 * Periodic rules (shared in meaning, not in code, with the CUDA side):
 *   wrap:          x <- x - L*floor(x/L); if x < 0 then x <- x + L;
 *                  if x >= L then x <- x - L
 *   minimum image: d = x_j - x_i; if d > L/2 then d -= L
 *                                 else if d < -L/2 then d += L
 *   list test:     dx*dx + dy*dy + dz*dz < rl*rl, left to right, rounded
 *                  after every operation (compiled with -ffp-contract=off).
 *
 * Units: A, eV, fs, u. 1 u (A/fs)^2 = 103.642696527 eV.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_RGL 0
#define ORC_SC 1
#define ORC_SPLINE 2

static const double ORC_MVV = 103.642696527;     /* eV per u (A/fs)^2 */
static const double ORC_KB = 8.617333262e-5;     /* eV/K */

/* ------------------------------------------------------------------ */
/* natural cubic spline on a uniform grid                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int n;            /* number of knots (>= 3) */
    double t0, h;     /* first knot, spacing */
    double* y;        /* knot values */
    double* m;        /* second derivatives, m[0] = m[n-1] = 0 */
} spline;

/* Second derivatives of the natural spline: tridiagonal system
 * (h/6) m[k-1] + (2h/3) m[k] + (h/6) m[k+1] = (y[k+1] - 2y[k] + y[k-1])/h,
 * m[0] = m[n-1] = 0, solved by the Thomas algorithm. */
static void spline_setup(spline* s) {
    int n = s->n;
    double h = s->h;
    double* c = (double*)calloc((size_t)n, sizeof(double));
    double* d = (double*)calloc((size_t)n, sizeof(double));
    s->m[0] = 0.0;
    s->m[n - 1] = 0.0;
    /* forward sweep over unknowns k = 1..n-2 */
    for (int k = 1; k <= n - 2; ++k) {
        double a = h / 6.0, b = 2.0 * h / 3.0, cc = h / 6.0;
        double rhs = (s->y[k + 1] - 2.0 * s->y[k] + s->y[k - 1]) / h;
        if (k == 1) {
            c[k] = cc / b;
            d[k] = rhs / b;
        } else {
            double den = b - a * c[k - 1];
            c[k] = cc / den;
            d[k] = (rhs - a * d[k - 1]) / den;
        }
    }
    for (int k = n - 2; k >= 1; --k) {
        s->m[k] = d[k] - (k < n - 2 ? c[k] * s->m[k + 1] : 0.0);
    }
    free(c);
    free(d);
}

/* value, first and second derivative at t; linear outside [t0, t_{n-1}] */
static void spline_eval(const spline* s, double t, double* v, double* d1, double* d2) {
    int n = s->n;
    double h = s->h;
    double tn = s->t0 + h * (n - 1);
    if (t < s->t0 || t > tn) {
        double te = t < s->t0 ? s->t0 : tn;
        double v0, s0, dd;
        spline_eval(s, te, &v0, &s0, &dd);
        *v = v0 + s0 * (t - te);
        *d1 = s0;
        *d2 = 0.0;
        return;
    }
    int k = (int)floor((t - s->t0) / h);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double tk = s->t0 + h * k;
    double B = (t - tk) / h;
    double A = 1.0 - B;
    double yk = s->y[k], yk1 = s->y[k + 1], mk = s->m[k], mk1 = s->m[k + 1];
    *v = A * yk + B * yk1 + ((A * A * A - A) * mk + (B * B * B - B) * mk1) * h * h / 6.0;
    *d1 = (yk1 - yk) / h - (3.0 * A * A - 1.0) / 6.0 * h * mk + (3.0 * B * B - 1.0) / 6.0 * h * mk1;
    *d2 = A * mk + B * mk1;
}

/* ------------------------------------------------------------------ */
/* potentials                                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind;
    double prm[8];
    double r_taper, r_cut;
    spline sp_phi, sp_f, sp_F;
    /* several species (splines only, Eq. 1-3 with the type labels a, b):
     * V^(ab) and rho^(ab) for each unordered pair a <= b (symmetric, as the
     * common factor (F'_i + F'_j) of Eq. (3) requires), F^(a) for each type;
     * one species uses sp_phi, sp_f, sp_F */
    int n_types;
    spline *aphi, *af, *aF;
    const int* types; /* per-atom species of the current call (orc_pot_set_types) */
} orc_pot;

/* index of the unordered type pair (a, b), a, b < T: row-major upper triangle */
static int pair_index(int T, int a, int b) {
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
    return a * T - a * (a - 1) / 2 + (b - a);
}

orc_pot* orc_pot_new(int kind, const double* prm, double r_taper, double r_cut, int n_phi, int n_f, int n_F,
                     const double* knots, double r_lo, double r_hi, double rho_lo, double rho_hi) {
    orc_pot* P = (orc_pot*)calloc(1, sizeof(orc_pot));
    P->kind = kind;
    for (int k = 0; k < 8; ++k) P->prm[k] = prm ? prm[k] : 0.0;
    P->r_taper = r_taper;
    P->r_cut = r_cut;
    if (kind == ORC_SPLINE) {
        spline* sps[3] = {&P->sp_phi, &P->sp_f, &P->sp_F};
        int ns[3] = {n_phi, n_f, n_F};
        const double* src = knots;
        for (int s = 0; s < 3; ++s) {
            sps[s]->n = ns[s];
            sps[s]->y = (double*)malloc(sizeof(double) * (size_t)ns[s]);
            sps[s]->m = (double*)malloc(sizeof(double) * (size_t)ns[s]);
            memcpy(sps[s]->y, src, sizeof(double) * (size_t)ns[s]);
            src += ns[s];
        }
        P->sp_phi.t0 = r_lo;
        P->sp_phi.h = (r_hi - r_lo) / (n_phi - 1);
        P->sp_f.t0 = r_lo;
        P->sp_f.h = (r_hi - r_lo) / (n_f - 1);
        P->sp_F.t0 = rho_lo;
        P->sp_F.h = (rho_hi - rho_lo) / (n_F - 1);
        for (int s = 0; s < 3; ++s) spline_setup(sps[s]);
        P->r_cut = r_hi;
        P->r_taper = r_hi;
    }
    P->n_types = 1;
    P->aphi = &P->sp_phi;
    P->af = &P->sp_f;
    P->aF = &P->sp_F;
    return P;
}

static void spline_from(spline* s, int n, const double* y, double t0, double t_end) {
    s->n = n;
    s->y = (double*)malloc(sizeof(double) * (size_t)n);
    s->m = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(s->y, y, sizeof(double) * (size_t)n);
    s->t0 = t0;
    s->h = (t_end - t0) / (n - 1);
    spline_setup(s);
}

/* Spline potential of n_types species. knots: V^(ab) for the P = T(T+1)/2
 * unordered pairs in pair_index order (n_r values each over [r_lo, r_hi]),
 * then rho^(ab) for the same pairs, then F^(a) for each type (n_rho values
 * each over [rho_lo, rho_hi]). r_cut = r_hi. */
orc_pot* orc_pot_new_alloy(int n_types, int n_r, int n_rho, const double* knots, double r_lo, double r_hi,
                           double rho_lo, double rho_hi) {
    orc_pot* P = (orc_pot*)calloc(1, sizeof(orc_pot));
    int np = n_types * (n_types + 1) / 2;
    P->kind = ORC_SPLINE;
    P->r_cut = r_hi;
    P->r_taper = r_hi;
    P->n_types = n_types;
    P->aphi = (spline*)calloc((size_t)np, sizeof(spline));
    P->af = (spline*)calloc((size_t)np, sizeof(spline));
    P->aF = (spline*)calloc((size_t)n_types, sizeof(spline));
    const double* src = knots;
    for (int k = 0; k < np; ++k, src += n_r) spline_from(&P->aphi[k], n_r, src, r_lo, r_hi);
    for (int k = 0; k < np; ++k, src += n_r) spline_from(&P->af[k], n_r, src, r_lo, r_hi);
    for (int k = 0; k < n_types; ++k, src += n_rho) spline_from(&P->aF[k], n_rho, src, rho_lo, rho_hi);
    /* the single-species fields mirror the (0, 0) tables for the callers
     * that ask for a table without types */
    P->sp_phi = P->aphi[0];
    P->sp_f = P->af[0];
    P->sp_F = P->aF[0];
    return P;
}

/* the per-atom species used by the following force calls (NULL: all 0);
 * the array stays owned by the caller */
void orc_pot_set_types(orc_pot* P, const int* types) { P->types = types; }

void orc_pot_free(orc_pot* P) {
    if (!P) return;
    if (P->kind == ORC_SPLINE && P->n_types > 1) {
        int np = P->n_types * (P->n_types + 1) / 2;
        for (int k = 0; k < np; ++k) {
            free(P->aphi[k].y); free(P->aphi[k].m);
            free(P->af[k].y); free(P->af[k].m);
        }
        for (int k = 0; k < P->n_types; ++k) {
            free(P->aF[k].y); free(P->aF[k].m);
        }
        free(P->aphi);
        free(P->af);
        free(P->aF);
    } else if (P->kind == ORC_SPLINE) {
        free(P->sp_phi.y); free(P->sp_phi.m);
        free(P->sp_f.y); free(P->sp_f.m);
        free(P->sp_F.y); free(P->sp_F.m);
    }
    free(P);
}

/* type-pair table of atoms i, j and type of atom i for the current types */
static int ptype(const orc_pot* P, int i, int j) {
    if (P->n_types <= 1 || !P->types) return 0;
    return pair_index(P->n_types, P->types[i], P->types[j]);
}
static int atype(const orc_pot* P, int i) { return P->n_types <= 1 || !P->types ? 0 : P->types[i]; }

/* C2 smoothstep taper and its derivative */
static void taper(double r, double rs, double rc, double* S, double* dS) {
    if (r <= rs || rs >= rc) {
        *S = r < rc ? 1.0 : 0.0;
        *dS = 0.0;
        return;
    }
    if (r >= rc) {
        *S = 0.0;
        *dS = 0.0;
        return;
    }
    double w = rc - rs;
    double x = (r - rs) / w;
    double x2 = x * x, x3 = x2 * x;
    *S = 1.0 - 10.0 * x3 + 15.0 * x3 * x - 6.0 * x3 * x2;
    *dS = (-30.0 * x2 + 60.0 * x3 - 30.0 * x3 * x) / w;
}

/* pair function V (phi) and density function rho (f), with r-derivatives */
static void pair_eval(const orc_pot* P, int pt, double r, double* phi, double* dphi, double* f, double* df) {
    if (r >= P->r_cut) {
        *phi = *dphi = *f = *df = 0.0;
        return;
    }
    if (P->kind == ORC_RGL) {
        double A = P->prm[0], xi = P->prm[1], p = P->prm[2], q = P->prm[3], r0 = P->prm[4];
        double S, dS;
        taper(r, P->r_taper, P->r_cut, &S, &dS);
        double e1 = exp(-p * (r / r0 - 1.0));
        double e2 = exp(-2.0 * q * (r / r0 - 1.0));
        *phi = 2.0 * A * e1 * S;
        *dphi = 2.0 * A * e1 * (-p / r0 * S + dS);
        *f = xi * xi * e2 * S;
        *df = xi * xi * e2 * (-2.0 * q / r0 * S + dS);
    } else if (P->kind == ORC_SC) {
        double eps = P->prm[0], a = P->prm[2], n = P->prm[3], m = P->prm[4];
        double S, dS;
        taper(r, P->r_taper, P->r_cut, &S, &dS);
        double an = pow(a / r, n), am = pow(a / r, m);
        *phi = eps * an * S;
        *dphi = eps * an * (-n / r * S + dS);
        *f = am * S;
        *df = am * (-m / r * S + dS);
    } else {
        double d2;
        spline_eval(&P->aphi[pt], r, phi, dphi, &d2);
        spline_eval(&P->af[pt], r, f, df, &d2);
    }
}

/* embedding function F(rho), F'(rho), F''(rho) */
static void embed_eval(const orc_pot* P, int a, double rho, double* F, double* Fp, double* Fpp) {
    if (P->kind == ORC_SPLINE) {
        spline_eval(&P->aF[a], rho, F, Fp, Fpp);
        return;
    }
    if (rho <= 0.0) {
        *F = *Fp = *Fpp = 0.0;
        return;
    }
    double scale = P->kind == ORC_SC ? P->prm[1] * P->prm[0] : 1.0; /* c*eps for SC */
    double sq = sqrt(rho);
    *F = -scale * sq;
    *Fp = -0.5 * scale / sq;
    *Fpp = 0.25 * scale / (rho * sq);
}

void orc_pot_eval(const orc_pot* P, int n, const double* r, double* phi, double* dphi, double* f, double* df) {
    for (int k = 0; k < n; ++k) pair_eval(P, 0, r[k], phi + k, dphi + k, f + k, df + k);
}

void orc_embed_eval(const orc_pot* P, int n, const double* rho, double* F, double* Fp, double* Fpp) {
    for (int k = 0; k < n; ++k) embed_eval(P, 0, rho[k], F + k, Fp + k, Fpp + k);
}

/* ------------------------------------------------------------------ */
/* periodic geometry                                                   */
/* ------------------------------------------------------------------ */

/* x - L*floor(x/L) can round to a tiny negative value (x just below k*L,
 * |k| >= 2, where L*k rounds above x) or to L; both are folded into [0, L). */
static double wrap1(double x, double L) {
    double y = x - L * floor(x / L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

static double minimg(double d, double L) {
    double h = 0.5 * L;
    if (d > h) return d - L;
    if (d < -h) return d + L;
    return d;
}

/* minimum-image separation d = x_j - x_i and its squared length */
static double sep(const double* x, int i, int j, const double* box, double* d) {
    d[0] = minimg(x[3 * j + 0] - x[3 * i + 0], box[0]);
    d[1] = minimg(x[3 * j + 1] - x[3 * i + 1], box[1]);
    d[2] = minimg(x[3 * j + 2] - x[3 * i + 2], box[2]);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

void orc_wrap(int n, double* x, const double* box) {
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) x[3 * i + a] = wrap1(x[3 * i + a], box[a]);
}

/* ------------------------------------------------------------------ */
/* neighbour pairs (half list, i < j)                                  */
/* ------------------------------------------------------------------ */

/* All pairs i<j with minimum-image r^2 < rl^2, by direct enumeration.
 * Returns the pair count; writes at most cap pairs. */
long orc_pairs_brute(int n, const double* x, const double* box, double rl, int* pi, int* pj, long cap) {
    double rl2 = rl * rl, d[3];
    long np = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            if (sep(x, i, j, box, d) < rl2) {
                if (np < cap) {
                    pi[np] = i;
                    pj[np] = j;
                }
                ++np;
            }
        }
    return np;
}

/* The same pair set by linked cells (Sec. 3.2): the box is cut into
 * NC(1) x NC(2) x NC(3) cells of side >= rl, each atom is chained into the
 * list of its cell (head/next arrays), and the candidates of an atom are the
 * atoms of its own cell and of the 26 neighbouring cells (periodic). Falls
 * back to direct enumeration when a dimension has fewer than 3 cells, where
 * the 26 neighbours would not be distinct. */
long orc_pairs_cells(int n, const double* x, const double* box, double rl, int* pi, int* pj, long cap) {
    int nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = (int)floor(box[a] / (rl * (1.0 + 1e-12)));
    if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3) return orc_pairs_brute(n, x, box, rl, pi, pj, cap);
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * (size_t)ncell);
    int* next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(x[3 * i + a] / (box[a] / nc[a]));
            if (c < 0) c = 0;
            if (c >= nc[a]) c = nc[a] - 1;
            ci[a] = c;
        }
        long c = ((long)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[i] = head[c];
        head[c] = i;
    }
    double rl2 = rl * rl, d[3];
    long np = 0;
    for (int cx = 0; cx < nc[0]; ++cx)
        for (int cy = 0; cy < nc[1]; ++cy)
            for (int cz = 0; cz < nc[2]; ++cz) {
                long c = ((long)cx * nc[1] + cy) * nc[2] + cz;
                for (int ox = -1; ox <= 1; ++ox)
                    for (int oy = -1; oy <= 1; ++oy)
                        for (int oz = -1; oz <= 1; ++oz) {
                            int qx = (cx + ox + nc[0]) % nc[0];
                            int qy = (cy + oy + nc[1]) % nc[1];
                            int qz = (cz + oz + nc[2]) % nc[2];
                            long q = ((long)qx * nc[1] + qy) * nc[2] + qz;
                            for (int i = head[c]; i >= 0; i = next[i])
                                for (int j = head[q]; j >= 0; j = next[j]) {
                                    if (i >= j) continue;
                                    if (sep(x, i, j, box, d) < rl2) {
                                        if (np < cap) {
                                            pi[np] = i;
                                            pj[np] = j;
                                        }
                                        ++np;
                                    }
                                }
                        }
            }
    free(head);
    free(next);
    return np;
}

/* ------------------------------------------------------------------ */
/* energies and forces                                                 */
/* ------------------------------------------------------------------ */

/* Eq. (1)-(3) written out as double sums over all ordered pairs j != i.
 * rho, e_atom: [n]; f: [n*3]. Returns E_T. Any output may be NULL. */
double orc_forces_brute(const orc_pot* P, int n, const double* x, const double* box, double* rho_out,
                        double* e_out, double* f_out) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rc2 = P->r_cut * P->r_cut;
    double* rho = (double*)calloc(nn, sizeof(double));
    double* Fp = (double*)calloc(nn, sizeof(double));
    double d[3], phi, dphi, f, df, F, Fpp;
    /* rho_i = sum_{j != i} rho(r_ij) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = sep(x, i, j, box, d);
            if (r2 >= rc2) continue;
            pair_eval(P, ptype(P, i, j), sqrt(r2), &phi, &dphi, &f, &df);
            rho[i] += f;
        }
    /* E_i = F(rho_i) + 1/2 sum_{j != i} V(r_ij);  E_T = sum_i E_i */
    double E = 0.0;
    for (int i = 0; i < n; ++i) {
        embed_eval(P, atype(P, i), rho[i], &F, &Fp[i], &Fpp);
        double e = F;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = sep(x, i, j, box, d);
            if (r2 >= rc2) continue;
            pair_eval(P, ptype(P, i, j), sqrt(r2), &phi, &dphi, &f, &df);
            e += 0.5 * phi;
        }
        if (e_out) e_out[i] = e;
        E += e;
    }
    /* f_i = -sum_j [(F'_i + F'_j) rho'(r) + V'(r)] r_ij / r, r_ij = x_i - x_j */
    if (f_out) {
        for (int i = 0; i < n; ++i) {
            double fi[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double r2 = sep(x, i, j, box, d); /* d = x_j - x_i = -r_ij */
                if (r2 >= rc2) continue;
                double r = sqrt(r2);
                pair_eval(P, ptype(P, i, j), r, &phi, &dphi, &f, &df);
                double w = (Fp[i] + Fp[j]) * df + dphi;
                for (int a = 0; a < 3; ++a) fi[a] -= w * (-d[a]) / r;
            }
            for (int a = 0; a < 3; ++a) f_out[3 * i + a] = fi[a];
        }
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    free(rho);
    free(Fp);
    return E;
}

/* The same quantities from a half list of pairs i<j (within the list
 * radius), each pair visited once and its force applied to both atoms with
 * opposite signs (Newton's third law), in two passes: densities, then
 * forces. rho, Fp, e_atom: [n]; f: [n*3]; any may be NULL. Returns E_T. */
double orc_forces_pairs(const orc_pot* P, int n, const double* x, const double* box, long np, const int* pi,
                        const int* pj, double* rho_out, double* Fp_out, double* e_out, double* f_out) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rc2 = P->r_cut * P->r_cut;
    double* rho = (double*)calloc(nn, sizeof(double));
    double* Fp = (double*)calloc(nn, sizeof(double));
    double* e = (double*)calloc(nn, sizeof(double));
    double* f = (double*)calloc(nn * 3, sizeof(double));
    double d[3], phi, dphi, fr, dfr, F, Fpp;
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        pair_eval(P, ptype(P, i, j), sqrt(r2), &phi, &dphi, &fr, &dfr);
        rho[i] += fr;
        rho[j] += fr;
    }
    for (int i = 0; i < n; ++i) {
        embed_eval(P, atype(P, i), rho[i], &F, &Fp[i], &Fpp);
        e[i] = F;
    }
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        double r = sqrt(r2);
        pair_eval(P, ptype(P, i, j), r, &phi, &dphi, &fr, &dfr);
        e[i] += 0.5 * phi;
        e[j] += 0.5 * phi;
        double s = dphi + (Fp[i] + Fp[j]) * dfr; /* dE_T / dr for this pair */
        for (int a = 0; a < 3; ++a) {
            double c = s * d[a] / r;
            f[3 * i + a] += c;
            f[3 * j + a] -= c;
        }
    }
    double E = 0.0;
    for (int i = 0; i < n; ++i) E += e[i];
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (Fp_out) memcpy(Fp_out, Fp, sizeof(double) * (size_t)n);
    if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)n);
    if (f_out) memcpy(f_out, f, sizeof(double) * 3 * (size_t)n);
    free(rho);
    free(Fp);
    free(e);
    free(f);
    return E;
}

/* ------------------------------------------------------------------ */
/* all-cores variants (CPU-baseline timing)                            */
/* ------------------------------------------------------------------ */

/* Threads used by orc_md_run for its pair list and force sums; 1 (the
 * default) runs the plain serial functions above. */
static int orc_threads = 1;

int orc_set_threads(int t) {
#ifdef _OPENMP
    orc_threads = t < 1 ? 1 : t;
#else
    (void)t;
    orc_threads = 1;
#endif
    return orc_threads;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_id(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

typedef struct {
    int* a;
    int* b;
    long n, cap;
} pairvec;

static void pv_push(pairvec* v, int i, int j) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 4096;
        v->a = (int*)realloc(v->a, sizeof(int) * (size_t)v->cap);
        v->b = (int*)realloc(v->b, sizeof(int) * (size_t)v->cap);
    }
    v->a[v->n] = i;
    v->b[v->n] = j;
    ++v->n;
}

/* orc_pairs_cells with its loop over cells cut into `threads` contiguous
 * slabs of the first cell index, each thread appending to its own buffer;
 * the buffers are joined in slab order, so the list (pairs and their order)
 * is that of orc_pairs_cells for any thread count. */
long orc_pairs_cells_par(int n, const double* x, const double* box, double rl, int* pi, int* pj, long cap,
                         int threads) {
    int nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = (int)floor(box[a] / (rl * (1.0 + 1e-12)));
    if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3) return orc_pairs_brute(n, x, box, rl, pi, pj, cap);
    int T = threads < 1 ? 1 : threads;
    if (T > nc[0]) T = nc[0];
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * (size_t)ncell);
    int* next = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (long c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            int c = (int)floor(x[3 * i + a] / (box[a] / nc[a]));
            if (c < 0) c = 0;
            if (c >= nc[a]) c = nc[a] - 1;
            ci[a] = c;
        }
        long c = ((long)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[i] = head[c];
        head[c] = i;
    }
    double rl2 = rl * rl;
    pairvec* buf = (pairvec*)calloc((size_t)T, sizeof(pairvec));
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static, 1)
#endif
    for (int t = 0; t < T; ++t) {
        int c0 = (int)((long)nc[0] * t / T), c1 = (int)((long)nc[0] * (t + 1) / T);
        double d[3];
        for (int cx = c0; cx < c1; ++cx)
            for (int cy = 0; cy < nc[1]; ++cy)
                for (int cz = 0; cz < nc[2]; ++cz) {
                    long c = ((long)cx * nc[1] + cy) * nc[2] + cz;
                    for (int ox = -1; ox <= 1; ++ox)
                        for (int oy = -1; oy <= 1; ++oy)
                            for (int oz = -1; oz <= 1; ++oz) {
                                int qx = (cx + ox + nc[0]) % nc[0];
                                int qy = (cy + oy + nc[1]) % nc[1];
                                int qz = (cz + oz + nc[2]) % nc[2];
                                long q = ((long)qx * nc[1] + qy) * nc[2] + qz;
                                for (int i = head[c]; i >= 0; i = next[i])
                                    for (int j = head[q]; j >= 0; j = next[j]) {
                                        if (i >= j) continue;
                                        if (sep(x, i, j, box, d) < rl2) pv_push(&buf[t], i, j);
                                    }
                            }
                }
    }
    long np = 0;
    for (int t = 0; t < T; ++t) {
        for (long k = 0; k < buf[t].n; ++k, ++np)
            if (np < cap) {
                pi[np] = buf[t].a[k];
                pj[np] = buf[t].b[k];
            }
        free(buf[t].a);
        free(buf[t].b);
    }
    free(buf);
    free(head);
    free(next);
    return np;
}

/* orc_forces_pairs over `threads` threads: the pair list is cut into
 * contiguous chunks, each thread sums its chunk into its own rho, E_i and
 * force arrays (thread 0's E_i start from F(rho_i), the others from 0), and
 * the partial arrays are added in thread order. One thread gives the
 * serial function's result bit for bit; more threads reorder the sums. */
double orc_forces_pairs_par(const orc_pot* P, int n, const double* x, const double* box, long np, const int* pi,
                            const int* pj, double* rho_out, double* Fp_out, double* e_out, double* f_out,
                            int threads) {
    int T = threads < 1 ? 1 : threads;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rc2 = P->r_cut * P->r_cut;
    double* rho_t = (double*)calloc(nn * (size_t)T, sizeof(double));
    double* e_t = (double*)calloc(nn * (size_t)T, sizeof(double));
    double* f_t = (double*)calloc(3 * nn * (size_t)T, sizeof(double));
    double* rho = (double*)calloc(nn, sizeof(double));
    double* Fp = (double*)calloc(nn, sizeof(double));
    double* e = (double*)calloc(nn, sizeof(double));
    double* f = (double*)calloc(3 * nn, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
    {
        int t = thread_id();
        long k0 = np * t / T, k1 = np * (t + 1) / T;
        int i0 = (int)((long)n * t / T), i1 = (int)((long)n * (t + 1) / T);
        double d[3], phi, dphi, fr, dfr, F, Fpp;
        double* rho_p = rho_t + nn * (size_t)t;
        double* e_p = e_t + nn * (size_t)t;
        double* f_p = f_t + 3 * nn * (size_t)t;
        for (long k = k0; k < k1; ++k) {
            int i = pi[k], j = pj[k];
            double r2 = sep(x, i, j, box, d);
            if (r2 >= rc2) continue;
            pair_eval(P, ptype(P, i, j), sqrt(r2), &phi, &dphi, &fr, &dfr);
            rho_p[i] += fr;
            rho_p[j] += fr;
        }
#ifdef _OPENMP
#pragma omp barrier
#endif
        for (int i = i0; i < i1; ++i) {
            double r = rho_t[i];
            for (int u = 1; u < T; ++u) r += rho_t[nn * (size_t)u + i];
            rho[i] = r;
            embed_eval(P, atype(P, i), r, &F, &Fp[i], &Fpp);
            e_t[i] = F; /* thread 0's E_i start from F(rho_i) */
        }
#ifdef _OPENMP
#pragma omp barrier
#endif
        for (long k = k0; k < k1; ++k) {
            int i = pi[k], j = pj[k];
            double r2 = sep(x, i, j, box, d);
            if (r2 >= rc2) continue;
            double r = sqrt(r2);
            pair_eval(P, ptype(P, i, j), r, &phi, &dphi, &fr, &dfr);
            e_p[i] += 0.5 * phi;
            e_p[j] += 0.5 * phi;
            double s = dphi + (Fp[i] + Fp[j]) * dfr;
            for (int a = 0; a < 3; ++a) {
                double c = s * d[a] / r;
                f_p[3 * i + a] += c;
                f_p[3 * j + a] -= c;
            }
        }
#ifdef _OPENMP
#pragma omp barrier
#endif
        for (int i = i0; i < i1; ++i) {
            double ei = e_t[i];
            for (int u = 1; u < T; ++u) ei += e_t[nn * (size_t)u + i];
            e[i] = ei;
            for (int a = 0; a < 3; ++a) {
                double fa = f_t[3 * i + a];
                for (int u = 1; u < T; ++u) fa += f_t[3 * nn * (size_t)u + 3 * i + a];
                f[3 * i + a] = fa;
            }
        }
    }
    double E = 0.0;
    for (int i = 0; i < n; ++i) E += e[i];
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (Fp_out) memcpy(Fp_out, Fp, sizeof(double) * (size_t)n);
    if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)n);
    if (f_out) memcpy(f_out, f, sizeof(double) * 3 * (size_t)n);
    free(rho_t);
    free(e_t);
    free(f_t);
    free(rho);
    free(Fp);
    free(e);
    free(f);
    return E;
}

/* Virial of the forces of Eq. (3) for the pressure of Eq. (6). The sum
 * W = sum_i f_i . r_i is written for a periodic box as a sum over pairs: the
 * forces are pairwise, f_ij = -f_ji with f_ij = -(dE_T/dr_ij) (r_i - r_j)/r_ij
 * (the bracket of Eq. (3) for the pair), so each pair i<j contributes
 * f_ij . (r_i - r_j) = -(dE_T/dr_ij) r_ij. Returns W in eV. */
double orc_virial_pairs(const orc_pot* P, int n, const double* x, const double* box, long np, const int* pi,
                        const int* pj) {
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rc2 = P->r_cut * P->r_cut;
    double* rho = (double*)calloc(nn, sizeof(double));
    double* Fp = (double*)calloc(nn, sizeof(double));
    double d[3], phi, dphi, fr, dfr, F, Fpp;
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        pair_eval(P, ptype(P, i, j), sqrt(r2), &phi, &dphi, &fr, &dfr);
        rho[i] += fr;
        rho[j] += fr;
    }
    for (int i = 0; i < n; ++i) embed_eval(P, atype(P, i), rho[i], &F, &Fp[i], &Fpp);
    double W = 0.0;
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        double r = sqrt(r2);
        pair_eval(P, ptype(P, i, j), r, &phi, &dphi, &fr, &dfr);
        W -= (dphi + (Fp[i] + Fp[j]) * dfr) * r;
    }
    free(rho);
    free(Fp);
    return W;
}

/* ------------------------------------------------------------------ */
/* velocity-Verlet dynamics                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    int* pi;
    int* pj;
    long np, cap;
} pairbuf;

static void pairs_rebuild(pairbuf* B, int n, const double* x, const double* box, double rl) {
    for (;;) {
        long np = orc_threads > 1 ? orc_pairs_cells_par(n, x, box, rl, B->pi, B->pj, B->cap, orc_threads)
                                  : orc_pairs_cells(n, x, box, rl, B->pi, B->pj, B->cap);
        if (np <= B->cap) {
            B->np = np;
            return;
        }
        B->cap = np + np / 4 + 16;
        B->pi = (int*)realloc(B->pi, sizeof(int) * (size_t)B->cap);
        B->pj = (int*)realloc(B->pj, sizeof(int) * (size_t)B->cap);
    }
}

/* forces and E_T of a step: the serial half-list sums, or their threaded
 * form when orc_set_threads asked for more than one thread */
static double step_forces(const orc_pot* P, int n, const double* x, const double* box, const pairbuf* B,
                          double* f) {
    if (orc_threads > 1)
        return orc_forces_pairs_par(P, n, x, box, B->np, B->pi, B->pj, NULL, NULL, NULL, f, orc_threads);
    return orc_forces_pairs(P, n, x, box, B->np, B->pi, B->pj, NULL, NULL, NULL, f);
}

static double kinetic(int n, const double* v, double mass) {
    double s = 0.0;
    for (int k = 0; k < 3 * n; ++k) s += v[k] * v[k];
    return 0.5 * mass * s * ORC_MVV;
}

/* Eq. (6): P = (N k_B T + W/3) / V with T the kinetic temperature (3n-3
 * degrees of freedom) and W the pair virial over the current list. */
static double pressure(const orc_pot* P, int n, const double* x, const double* v, const double* box, double mass,
                       const pairbuf* B) {
    double dof = 3.0 * n - 3.0;
    double T = dof > 0 ? 2.0 * kinetic(n, v, mass) / (dof * ORC_KB) : 0.0;
    double W = orc_virial_pairs(P, n, x, box, B->np, B->pi, B->pj);
    return (n * ORC_KB * T + W / 3.0) / (box[0] * box[1] * box[2]);
}

/* Electron-phonon friction of Finnis et al. (Eq. 4): each atom feels
 * -m (1/tau) (T_i - T_e)/T_i v_i, with T_i = m v_i^2 / (3 k_B) its own
 * kinetic temperature and T_e the constant electronic temperature. On its
 * own this term gives dT_i/dt = -(2/tau)(T_i - T_e) along the fixed direction
 * of v_i, which is integrated exactly over an interval h:
 *   T_i <- T_e + (T_i - T_e) exp(-2h/tau),  v_i <- v_i sqrt(T_i new / T_i old).
 * An atom at rest is left at rest (its direction is undefined). */
static void bath_half(int n, double* v, double mass, double T_e, double decay) {
    for (int i = 0; i < n; ++i) {
        double* vi = v + 3 * (size_t)i;
        double v2 = vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2];
        if (!(v2 > 0.0)) continue;
        double Ti = mass * ORC_MVV * v2 / (3.0 * ORC_KB);
        double Tn = T_e + (Ti - T_e) * decay;
        double lam = sqrt(Tn / Ti);
        vi[0] *= lam;
        vi[1] *= lam;
        vi[2] *= lam;
    }
}

/* n_steps of velocity Verlet at time step dt (fs) for atoms of one mass (u):
 *   [friction dt/2;] v += dt/2 * f/m;  x += dt * v;  wrap x;
 *   rebuild the list (radius r_cut + skin) when some atom moved more than
 *   skin/2 since the last build;
 *   f = forces(x);  v += dt/2 * f/m[; friction dt/2]
 *   [; pressure P of Eq. (6); x and box scaled by mu of Eq. (5)].
 * The bracketed friction half steps (Eq. 4, symmetric splitting) run when
 * tau_T > 0, towards the electronic temperature T_e (K). The bracketed
 * pressure coupling (Berendsen, Eq. 5) runs when tau_p > 0: with the
 * instantaneous pressure P = (N k_B T + W/3)/V (T the kinetic temperature
 * with 3n-3 degrees of freedom, W the pair virial), all coordinates and the
 * box lengths are multiplied by mu = [1 - beta (dt/tau_p)(P0 - P)]^(1/3),
 * beta the compressibility (A^3/eV), P0 the target (eV/A^3).
 * x, v: [n*3], updated in place; box: [3], updated in place when the
 * pressure is coupled. thermo (nullable): [(n_steps+1)*4] rows of (kinetic,
 * potential, total energy in eV, temperature in K with 3n-3 degrees of
 * freedom), row 0 the initial state, each row before that step's scaling.
 * press (nullable): [n_steps+1] the pressure of each row (eV/A^3). Returns
 * the number of list builds after the initial one. */
long orc_md_run(const orc_pot* P, int n, double* x, double* v, double* box, double mass, double dt,
                double skin, int n_steps, double* thermo, double tau_T, double T_e, double tau_p, double P0,
                double beta, double* press) {
    const int bath = tau_T > 0.0;
    const double decay = bath ? exp(-dt / tau_T) : 1.0; /* exp(-2 (dt/2) / tau) */
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rl = P->r_cut + skin;
    double half2 = 0.25 * skin * skin;
    double acc = 1.0 / (mass * ORC_MVV); /* (A/fs^2) per (eV/A) */
    double dof = 3.0 * n - 3.0;
    pairbuf B = {NULL, NULL, 0, 0};
    double* xb = (double*)malloc(sizeof(double) * 3 * nn);
    double* f = (double*)calloc(3 * nn, sizeof(double));
    orc_wrap(n, x, box);
    pairs_rebuild(&B, n, x, box, rl);
    memcpy(xb, x, sizeof(double) * 3 * (size_t)n);
    double pe = step_forces(P, n, x, box, &B, f);
    long rebuilds = 0;
    if (thermo) {
        double ke = kinetic(n, v, mass);
        thermo[0] = ke;
        thermo[1] = pe;
        thermo[2] = ke + pe;
        thermo[3] = dof > 0 ? 2.0 * ke / (dof * ORC_KB) : 0.0;
    }
    if (press) press[0] = pressure(P, n, x, v, box, mass, &B);
    for (int s = 1; s <= n_steps; ++s) {
        if (bath) bath_half(n, v, mass, T_e, decay);
        for (int k = 0; k < 3 * n; ++k) {
            v[k] += 0.5 * dt * f[k] * acc;
            x[k] += dt * v[k];
        }
        orc_wrap(n, x, box);
        double dmax2 = 0.0;
        for (int i = 0; i < n; ++i) {
            double dd = 0.0;
            for (int a = 0; a < 3; ++a) {
                double q = minimg(x[3 * i + a] - xb[3 * i + a], box[a]);
                dd += q * q;
            }
            if (dd > dmax2) dmax2 = dd;
        }
        if (dmax2 > half2) {
            pairs_rebuild(&B, n, x, box, rl);
            memcpy(xb, x, sizeof(double) * 3 * (size_t)n);
            ++rebuilds;
        }
        pe = step_forces(P, n, x, box, &B, f);
        for (int k = 0; k < 3 * n; ++k) v[k] += 0.5 * dt * f[k] * acc;
        if (bath) bath_half(n, v, mass, T_e, decay);
        if (thermo) {
            double ke = kinetic(n, v, mass);
            double* t = thermo + 4 * (size_t)s;
            t[0] = ke;
            t[1] = pe;
            t[2] = ke + pe;
            t[3] = dof > 0 ? 2.0 * ke / (dof * ORC_KB) : 0.0;
        }
        if (press || tau_p > 0.0) {
            double p_now = pressure(P, n, x, v, box, mass, &B);
            if (press) press[s] = p_now;
            if (tau_p > 0.0) {
                double mu = cbrt(1.0 - beta * (dt / tau_p) * (P0 - p_now));
                for (int k = 0; k < 3 * n; ++k) x[k] *= mu;
                for (int a = 0; a < 3; ++a) box[a] *= mu;
            }
        }
    }
    free(B.pi);
    free(B.pj);
    free(xb);
    free(f);
    return rebuilds;
}

/* ------------------------------------------------------------------ */
/* parameter derivatives by forward-mode dual numbers                  */
/* ------------------------------------------------------------------ */

/* A dual number v + d*eps carries one directional derivative through the
 * same formulas as above; seeding one parameter's d = 1 gives the exact
 * derivative of every rho_i, F_i and E_T with respect to it. */
typedef struct {
    double v, d;
} dual;

static dual dc(double v) { dual r = {v, 0.0}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.d - b.d}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual ddiv(dual a, dual b) {
    dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
    return r;
}
static dual dscale(dual a, double s) { dual r = {a.v * s, a.d * s}; return r; }
static dual dexp(dual a) { double e = exp(a.v); dual r = {e, e * a.d}; return r; }
static dual dsqrt(dual a) { double s = sqrt(a.v); dual r = {s, 0.5 * a.d / s}; return r; }
static dual dlog(dual a) { dual r = {log(a.v), a.d / a.v}; return r; }
/* b^e for b > 0, both dual: exp(e log b) */
static dual dpow(dual b, dual e) { return dexp(dmul(e, dlog(b))); }

typedef struct {
    int n;
    double t0, h;
    dual* y;
    dual* m;
} dspline;

static void dspline_setup(dspline* s) {
    int n = s->n;
    double h = s->h;
    dual* c = (dual*)calloc((size_t)n, sizeof(dual));
    dual* d = (dual*)calloc((size_t)n, sizeof(dual));
    s->m[0] = dc(0.0);
    s->m[n - 1] = dc(0.0);
    for (int k = 1; k <= n - 2; ++k) {
        double a = h / 6.0, b = 2.0 * h / 3.0, cc = h / 6.0;
        dual rhs = dscale(dadd(dsub(s->y[k + 1], dscale(s->y[k], 2.0)), s->y[k - 1]), 1.0 / h);
        if (k == 1) {
            c[k] = dc(cc / b);
            d[k] = dscale(rhs, 1.0 / b);
        } else {
            double den = b - a * c[k - 1].v; /* the matrix holds no parameter */
            c[k] = dc(cc / den);
            d[k] = dscale(dsub(rhs, dscale(d[k - 1], a)), 1.0 / den);
        }
    }
    for (int k = n - 2; k >= 1; --k) s->m[k] = k < n - 2 ? dsub(d[k], dscale(s->m[k + 1], c[k].v)) : d[k];
    free(c);
    free(d);
}

static void dspline_eval(const dspline* s, dual t, dual* v, dual* d1) {
    int n = s->n;
    double h = s->h;
    double tn = s->t0 + h * (n - 1);
    if (t.v < s->t0 || t.v > tn) {
        dual te = dc(t.v < s->t0 ? s->t0 : tn);
        dual v0, s0;
        dspline_eval(s, te, &v0, &s0);
        *v = dadd(v0, dmul(s0, dsub(t, te)));
        *d1 = s0;
        return;
    }
    int k = (int)floor((t.v - s->t0) / h);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double tk = s->t0 + h * k;
    dual B = dscale(dsub(t, dc(tk)), 1.0 / h);
    dual A = dsub(dc(1.0), B);
    dual A3 = dsub(dmul(dmul(A, A), A), A), B3 = dsub(dmul(dmul(B, B), B), B);
    *v = dadd(dadd(dmul(A, s->y[k]), dmul(B, s->y[k + 1])),
              dscale(dadd(dmul(A3, s->m[k]), dmul(B3, s->m[k + 1])), h * h / 6.0));
    dual a2 = dscale(dsub(dscale(dmul(A, A), 3.0), dc(1.0)), h / 6.0);
    dual b2 = dscale(dsub(dscale(dmul(B, B), 3.0), dc(1.0)), h / 6.0);
    *d1 = dadd(dsub(dscale(dsub(s->y[k + 1], s->y[k]), 1.0 / h), dmul(a2, s->m[k])), dmul(b2, s->m[k + 1]));
}

typedef struct {
    int kind;
    dual prm[8];
    double r_taper, r_cut;
    dspline sp[3]; /* phi, f, F (one species) */
    /* several species: P V tables, P rho tables, T F tables (as orc_pot) */
    int n_types, n_tab;
    dspline* tab;
} dpot;

/* Builds the dual potential with parameter `which` seeded (d = 1).
 * RGL order: A, xi, p, q, r0. Sutton-Chen order: eps, c, a, n, m.
 * Spline order: phi knots, f knots, F knots. */
static void dpot_init(dpot* D, const orc_pot* P, int which) {
    D->kind = P->kind;
    D->r_taper = P->r_taper;
    D->r_cut = P->r_cut;
    D->n_types = P->n_types;
    D->n_tab = 0;
    D->tab = NULL;
    for (int k = 0; k < 8; ++k) D->prm[k] = dc(P->prm[k]);
    if (P->kind != ORC_SPLINE) {
        if (which >= 0 && which < 8) D->prm[which].d = 1.0;
        return;
    }
    if (P->n_types > 1) {
        /* the tables in knot order: V pairs, rho pairs, F types */
        int np = P->n_types * (P->n_types + 1) / 2;
        D->n_tab = 2 * np + P->n_types;
        D->tab = (dspline*)calloc((size_t)D->n_tab, sizeof(dspline));
        int base = 0;
        for (int t = 0; t < D->n_tab; ++t) {
            const spline* src = t < np ? &P->aphi[t] : (t < 2 * np ? &P->af[t - np] : &P->aF[t - 2 * np]);
            dspline* dst = &D->tab[t];
            dst->n = src->n;
            dst->t0 = src->t0;
            dst->h = src->h;
            dst->y = (dual*)malloc(sizeof(dual) * (size_t)src->n);
            dst->m = (dual*)malloc(sizeof(dual) * (size_t)src->n);
            for (int k = 0; k < src->n; ++k) dst->y[k] = dc(src->y[k]);
            if (which >= base && which < base + src->n) dst->y[which - base].d = 1.0;
            base += src->n;
            dspline_setup(dst);
        }
        return;
    }
    const spline* src[3] = {&P->sp_phi, &P->sp_f, &P->sp_F};
    int base = 0;
    for (int s = 0; s < 3; ++s) {
        D->sp[s].n = src[s]->n;
        D->sp[s].t0 = src[s]->t0;
        D->sp[s].h = src[s]->h;
        D->sp[s].y = (dual*)malloc(sizeof(dual) * (size_t)src[s]->n);
        D->sp[s].m = (dual*)malloc(sizeof(dual) * (size_t)src[s]->n);
        for (int k = 0; k < src[s]->n; ++k) D->sp[s].y[k] = dc(src[s]->y[k]);
        if (which >= base && which < base + src[s]->n) D->sp[s].y[which - base].d = 1.0;
        base += src[s]->n;
        dspline_setup(&D->sp[s]);
    }
}

static void dpot_free(dpot* D) {
    if (D->kind != ORC_SPLINE) return;
    if (D->tab) {
        for (int t = 0; t < D->n_tab; ++t) {
            free(D->tab[t].y);
            free(D->tab[t].m);
        }
        free(D->tab);
        return;
    }
    for (int s = 0; s < 3; ++s) {
        free(D->sp[s].y);
        free(D->sp[s].m);
    }
}

static void dpair_eval(const dpot* D, int pt, double r, dual* phi, dual* dphi, dual* f, dual* df) {
    if (r >= D->r_cut) {
        *phi = *dphi = *f = *df = dc(0.0);
        return;
    }
    if (D->kind == ORC_RGL) {
        dual A = D->prm[0], xi = D->prm[1], p = D->prm[2], q = D->prm[3], r0 = D->prm[4];
        double S, dS;
        taper(r, D->r_taper, D->r_cut, &S, &dS);
        dual u = dsub(ddiv(dc(r), r0), dc(1.0));
        dual e1 = dexp(dscale(dmul(p, u), -1.0));
        dual e2 = dexp(dscale(dmul(q, u), -2.0));
        dual a2 = dscale(dmul(A, e1), 2.0);
        dual xi2 = dmul(xi, xi);
        *phi = dscale(a2, S);
        *dphi = dmul(a2, dadd(dscale(ddiv(p, r0), -S), dc(dS)));
        *f = dscale(dmul(xi2, e2), S);
        *df = dmul(dmul(xi2, e2), dadd(dscale(ddiv(q, r0), -2.0 * S), dc(dS)));
    } else if (D->kind == ORC_SC) {
        dual eps = D->prm[0], a = D->prm[2], n = D->prm[3], m = D->prm[4];
        double S, dS;
        taper(r, D->r_taper, D->r_cut, &S, &dS);
        dual ar = ddiv(a, dc(r));
        dual an = dpow(ar, n), am = dpow(ar, m);
        dual ean = dmul(eps, an);
        *phi = dscale(ean, S);
        *dphi = dmul(ean, dadd(dscale(ddiv(n, dc(r)), -S), dc(dS)));
        *f = dscale(am, S);
        *df = dmul(am, dadd(dscale(ddiv(m, dc(r)), -S), dc(dS)));
    } else if (D->tab) {
        int np = D->n_types * (D->n_types + 1) / 2;
        dspline_eval(&D->tab[pt], dc(r), phi, dphi);
        dspline_eval(&D->tab[np + pt], dc(r), f, df);
    } else {
        dspline_eval(&D->sp[0], dc(r), phi, dphi);
        dspline_eval(&D->sp[1], dc(r), f, df);
    }
}

static void dembed_eval(const dpot* D, int a, dual rho, dual* F, dual* Fp) {
    if (D->kind == ORC_SPLINE) {
        if (D->tab)
            dspline_eval(&D->tab[D->n_types * (D->n_types + 1) + a], rho, F, Fp);
        else
            dspline_eval(&D->sp[2], rho, F, Fp);
        return;
    }
    if (rho.v <= 0.0) {
        *F = *Fp = dc(0.0);
        return;
    }
    /* F = -scale sqrt(rho): scale 1 for RGL, c*eps for Sutton-Chen */
    dual scale = D->kind == ORC_SC ? dmul(D->prm[1], D->prm[0]) : dc(1.0);
    dual sq = dsqrt(rho);
    *F = dscale(dmul(scale, sq), -1.0);
    *Fp = ddiv(dscale(scale, -0.5), sq);
}

/* Directional derivatives of the forces and the energy of one configuration
 * with respect to parameter `which`: dF [n*3] = dF_i/dtheta, returns dE_T/dtheta.
 * Pairs are a half list as for orc_forces_pairs. */
double orc_param_deriv(const orc_pot* P, int which, int n, const double* x, const double* box, long np,
                       const int* pi, const int* pj, double* dF) {
    dpot D;
    dpot_init(&D, P, which);
    size_t nn = (size_t)(n > 0 ? n : 1);
    double rc2 = D.r_cut * D.r_cut;
    dual* rho = (dual*)calloc(nn, sizeof(dual));
    dual* Fp = (dual*)calloc(nn, sizeof(dual));
    dual E = dc(0.0);
    double d[3];
    dual phi, dphi, fr, dfr, F;
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        dpair_eval(&D, ptype(P, i, j), sqrt(r2), &phi, &dphi, &fr, &dfr);
        rho[i] = dadd(rho[i], fr);
        rho[j] = dadd(rho[j], fr);
    }
    for (int i = 0; i < n; ++i) {
        dembed_eval(&D, atype(P, i), rho[i], &F, &Fp[i]);
        E = dadd(E, F);
    }
    for (int k = 0; k < 3 * n; ++k) dF[k] = 0.0;
    for (long k = 0; k < np; ++k) {
        int i = pi[k], j = pj[k];
        double r2 = sep(x, i, j, box, d);
        if (r2 >= rc2) continue;
        double r = sqrt(r2);
        dpair_eval(&D, ptype(P, i, j), r, &phi, &dphi, &fr, &dfr);
        E = dadd(E, phi);
        dual s = dadd(dphi, dmul(dadd(Fp[i], Fp[j]), dfr));
        for (int a = 0; a < 3; ++a) {
            double c = s.d * d[a] / r;
            dF[3 * i + a] += c;
            dF[3 * j + a] -= c;
        }
    }
    free(rho);
    free(Fp);
    dpot_free(&D);
    return E.d;
}

/* Gradient of a scalar loss with respect to every parameter of the
 * potential, for one configuration, given gF = dL/dF_i [n*3] and
 * gE = dL/dE_T: grad[k] += sum_i gF_i . dF_i/dtheta_k + gE dE_T/dtheta_k.
 * n_param: 5 for RGL (A, xi, p, q, r0), n_phi + n_f + n_F for a spline. */
void orc_param_grad(const orc_pot* P, int n_param, int n, const double* x, const double* box, long np,
                    const int* pi, const int* pj, const double* gF, double gE, double* grad) {
    double* dF = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n_param; ++k) {
        double dE = orc_param_deriv(P, k, n, x, box, np, pi, pj, dF);
        double s = gE * dE;
        for (int q = 0; q < 3 * n; ++q) s += gF[q] * dF[q];
        grad[k] += s;
    }
    free(dF);
}
