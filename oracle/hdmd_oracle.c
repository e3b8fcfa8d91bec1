/*
 * hdmd_oracle.c -- plain, slow, FP64 CPU oracle for the hot path of
 * d-dimensional soft-sphere molecular dynamics (Hoy & Interiano-Alberto,
 * "Efficient d-dimensional molecular dynamics simulations for studies of the
 * glass-jamming transition", arXiv:2112.12271).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load or call this file.  The CUDA library
 * never links it, and the two share no code, header, table or constant.
 *
 * Everything here is double precision, serial and written for a reader who
 * wants to check it against the paper by eye:
 *   - minimum-image distances under periodic boundaries in all d axes
 *     (Sec. II.A, last paragraph; box centred at the origin);
 *   - Verlet lists two ways: brute force over all pairs (the plain
 *     definition) and the paper's linked-subcell loop nest (Sec. II.C, Fig. 1,
 *     Eqs. (7)-(9)); each checks the other;
 *   - the harmonic soft-sphere pair law U = (eps/2)(1 - r/s_ij)^2 for
 *     r < s_ij with s_ij = (s_i + s_j)/2 (the Lorentz mixing rule of
 *     Sec. II.A; the paper says the radial law is a user choice), or the
 *     paper's own truncated and shifted Morse law (Eq. (1)) with the
 *     volume-scaled prefactors eps_i = sigma_i^d mixed as sqrt(eps_i eps_j)
 *     (Sec. II.A), selected for every routine by orc_set_law;
 *   - the effective hard-sphere diameter of the Morse law (Eq. (12)) behind
 *     the packing fractions of Table III;
 *   - kick-drift-kick velocity Verlet (Sec. II.B);
 *   - FIRE 2.0 with the semi-implicit Euler integrator (Sec. II.B; the
 *     paper names the method but prints neither steps nor constants, so the
 *     steps follow the published FIRE 2.0 algorithm, see orc_fire);
 *   - serial SWAP Monte Carlo with Eqs. (10)-(11) (Sec. II.D);
 *   - the Philox4x32-10 counter-based generator (Salmon et al., SC'11) used
 *     to draw SWAP pairs and Metropolis uniforms from a seed.
 *
 * Readings of points the paper leaves open are stated at each function.
 * Positions are row-major x[i*d + k] with every coordinate in [-L/2, L/2).
 * Build with -ffp-contract=off so that x86 and Arm give the same bits.
 *
 * The tests use the serial build.  A second build with -fopenmp, used only
 * to time the oracle on all host cores, runs the per-atom loops (forces over
 * the lists, kicks and drift, the trigger) and the per-subcell loop of the
 * list build in parallel, as the paper's OpenMP code does (Sec. II); its
 * energy and virial sums may then differ from the serial ones in rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP build (1 in the serial build); returns the count
 * the build will use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define ORC_MAXD 16

/* ------------------------------------------------------------------ */
/* geometry                                                             */
/* ------------------------------------------------------------------ */

/* Volume of a d-dimensional sphere of diameter sigma, Eq. (2). */
double orc_sphere_volume(int d, double sigma)
{
    return pow(M_PI, 0.5 * d) * pow(sigma, d) / (pow(2.0, d) * tgamma(1.0 + 0.5 * d));
}

/* Subcells per axis, Eq. (7): floor(L / (largest diameter + skin)). */
int orc_n_cell(double L, double rc_max)
{
    return (int)floor(L / rc_max);
}

/* Linear subcell index of Eq. (9): I = sum_k C_k n^(d-k), axis 1 most
 * significant (k counts from 1 in the paper, from 0 here). */
int64_t orc_cell_index(int d, int n, const int *C)
{
    int64_t I = 0;
    for (int k = 0; k < d; ++k) I = I * n + C[k];
    return I;
}

/* Subcell coordinate of a position along one axis: the subcell whose
 * centre is given by Eq. (8).  Clamped against round-off at x = L/2. */
static int cell_coord(double x, double L, int n)
{
    double Lsc = L / n;
    int c = (int)floor((x + 0.5 * L) / Lsc);
    if (c < 0) c = 0;
    if (c > n - 1) c = n - 1;
    return c;
}

/* Minimum-image separation along one axis (periodic in every axis). */
double orc_min_image(double dx, double L)
{
    return dx - L * rint(dx / L);
}

/* Squared minimum-image distance between atoms i and j. */
static double dist2(int d, double L, const double *x, int64_t i, int64_t j)
{
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double dx = orc_min_image(x[j * d + k] - x[i * d + k], L);
        r2 += dx * dx;
    }
    return r2;
}

/* Verlet-list radius for the pair (i, j).  The paper's r_c^max is the
 * largest interaction range plus the skin (Sec. II.C).  Reading: the list
 * keeps a pair when r < s_ij + skin (per pair, mode 0) or r < s_max + skin
 * (one global radius, mode 1). */
static double list_radius(double si, double sj, double skin, int global_cut, double smax)
{
    return global_cut ? smax + skin : 0.5 * (si + sj) + skin;
}

static double max_of(const double *a, int64_t n)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (a[i] > m) m = a[i];
    return m;
}

/* ------------------------------------------------------------------ */
/* Verlet lists                                                         */
/* ------------------------------------------------------------------ */

/* Full Verlet lists by brute force over all pairs (the plain definition):
 * j is in VL(i) iff j != i and |x_j - x_i|^2 < rc_ij^2 with minimum image.
 * counts[N] receives the list lengths; when idx is non-NULL it receives the
 * lists back to back, each in ascending j, and must hold cap entries.
 * Returns the total number of entries, or -1 if idx is too small. */
int64_t orc_neighbors_brute(int d, int64_t N, double L, const double *x,
                            const double *sigma, double skin, int global_cut,
                            int32_t *counts, int32_t *idx, int64_t cap)
{
    double smax = max_of(sigma, N);
    int64_t tot = 0;
    for (int64_t i = 0; i < N; ++i) {
        int32_t c = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double rc = list_radius(sigma[i], sigma[j], skin, global_cut, smax);
            if (dist2(d, L, x, i, j) < rc * rc) {
                if (idx) {
                    if (tot >= cap) return -1;
                    idx[tot] = (int32_t)j;
                }
                ++tot;
                ++c;
            }
        }
        counts[i] = c;
    }
    return tot;
}

/* The list of one atom i by the same plain definition: every j != i whose
 * minimum-image distance is below the list radius, ascending.  For checking
 * sampled atoms of systems too large for the all-pairs routine.  Returns the
 * count (idx may be NULL to count only; -1 if the count exceeds cap). */
int64_t orc_neighbors_of(int d, int64_t N, double L, const double *x,
                         const double *sigma, double skin, int global_cut,
                         int64_t i, int32_t *idx, int64_t cap)
{
    double smax = max_of(sigma, N);
    int64_t c = 0;
    for (int64_t j = 0; j < N; ++j) {
        if (j == i) continue;
        double rc = list_radius(sigma[i], sigma[j], skin, global_cut, smax);
        if (dist2(d, L, x, i, j) < rc * rc) {
            if (idx) {
                if (c >= cap) return -1;
                idx[c] = (int32_t)j;
            }
            ++c;
        }
    }
    return c;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Full Verlet lists with the paper's linked-subcell loop nest (Sec. II.C,
 * Fig. 1): one outer loop over subcells I, the 3^d linked subcells of I
 * enumerated on the fly from a base-3 counter, then the double loop over
 * the atoms of I and of the linked subcell.  Reading for n_cell < 3: the
 * offsets -1 and +1 name the same subcell when n_cell = 2, so each distinct
 * subcell is visited once (offsets {0, +1}); n_cell must be >= 2, which
 * holds whenever L >= 2 (s_max + skin).  Output as orc_neighbors_brute,
 * each list sorted ascending.  Returns -2 if n_cell < 2. */
int64_t orc_neighbors_cells(int d, int64_t N, double L, const double *x,
                            const double *sigma, double skin, int global_cut,
                            int32_t *counts, int32_t *idx, int64_t cap)
{
    double smax = max_of(sigma, N);
    int n = orc_n_cell(L, smax + skin);
    if (n < 2) return -2;
    int64_t ncells = 1;
    for (int k = 0; k < d; ++k) ncells *= n;

    /* assign atoms to subcells (serial in the paper too) */
    int64_t *cell = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *head = malloc(sizeof(int64_t) * (size_t)(ncells + 1));
    int64_t *members = malloc(sizeof(int64_t) * (size_t)N);
    memset(head, 0, sizeof(int64_t) * (size_t)(ncells + 1));
    for (int64_t i = 0; i < N; ++i) {
        int C[ORC_MAXD];
        for (int k = 0; k < d; ++k) C[k] = cell_coord(x[i * d + k], L, n);
        cell[i] = orc_cell_index(d, n, C);
        head[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncells; ++c) head[c + 1] += head[c];
    {
        int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncells);
        memcpy(fill, head, sizeof(int64_t) * (size_t)ncells);
        for (int64_t i = 0; i < N; ++i) members[fill[cell[i]]++] = i;
        free(fill);
    }

    /* per-atom lists, collected in atom order afterwards */
    int32_t **lst = calloc((size_t)N, sizeof(int32_t *));
    int32_t *len = calloc((size_t)N, sizeof(int32_t));
    int32_t *capi = calloc((size_t)N, sizeof(int32_t));

    int64_t nstencil = 1;
    for (int k = 0; k < d; ++k) nstencil *= 3;

    /* one subcell per iteration; atom i's list is written only by the
     * iteration of its own subcell */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t I = 0; I < ncells; ++I) {
        int C[ORC_MAXD];
        int64_t rem = I;
        for (int k = d - 1; k >= 0; --k) { C[k] = (int)(rem % n); rem /= n; }
        for (int64_t s = 0; s < nstencil; ++s) {
            /* base-3 digits of s, axis 1 most significant: offset = digit-1 */
            int off[ORC_MAXD], skip = 0;
            int64_t t = s;
            for (int k = d - 1; k >= 0; --k) { off[k] = (int)(t % 3) - 1; t /= 3; }
            for (int k = 0; k < d; ++k)
                if (n == 2 && off[k] == -1) skip = 1; /* same subcell as +1 */
            if (skip) continue;
            int CJ[ORC_MAXD];
            for (int k = 0; k < d; ++k) CJ[k] = ((C[k] + off[k]) % n + n) % n;
            int64_t J = orc_cell_index(d, n, CJ);
            for (int64_t a = head[I]; a < head[I + 1]; ++a) {
                int64_t i = members[a];
                for (int64_t b = head[J]; b < head[J + 1]; ++b) {
                    int64_t j = members[b];
                    if (j == i) continue;
                    double rc = list_radius(sigma[i], sigma[j], skin, global_cut, smax);
                    if (dist2(d, L, x, i, j) < rc * rc) {
                        if (len[i] == capi[i]) {
                            capi[i] = capi[i] ? 2 * capi[i] : 16;
                            lst[i] = realloc(lst[i], sizeof(int32_t) * (size_t)capi[i]);
                        }
                        lst[i][len[i]++] = (int32_t)j;
                    }
                }
            }
        }
    }

    int64_t tot = 0;
    int overflow = 0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) qsort(lst[i], (size_t)len[i], sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < N; ++i) {
        counts[i] = len[i];
        if (idx) {
            if (tot + len[i] > cap) overflow = 1;
            else memcpy(idx + tot, lst[i], sizeof(int32_t) * (size_t)len[i]);
        }
        tot += len[i];
        free(lst[i]);
    }
    free(lst); free(len); free(capi); free(cell); free(head); free(members);
    return overflow ? -1 : tot;
}

/* ------------------------------------------------------------------ */
/* pair law, forces, energy, virial                                     */
/* ------------------------------------------------------------------ */

/* Harmonic soft spheres: U = (eps/2)(1 - r/s)^2 for r < s, else 0.  The
 * force on i from j is (eps/s)(1 - r/s) along (x_i - x_j)/r; *fr receives
 * that magnitude divided by r (0 at r = 0, a measure-zero guard).  Returns U. */
double orc_harmonic(double r, double s, double eps, double *fr)
{
    if (r >= s) { *fr = 0.0; return 0.0; }
    double g = 1.0 - r / s;
    *fr = (r > 0.0) ? (eps / s) * g / r : 0.0;
    return 0.5 * eps * g * g;
}

/* The truncated and shifted Morse law, Eq. (1):
 *   U(r) = eps [exp(-2a(r - s)) - 2 exp(-a(r - s)) + 1]   for r <= s,
 * and 0 for r >= s (the two agree at r = s, where U = 0).  Its force on i
 * from j is -dU/dr = eps [2a exp(-2a(r - s)) - 2a exp(-a(r - s))] along
 * (x_i - x_j)/r; *fr receives that magnitude divided by r. */
double orc_morse(double r, double s, double eps, double a, double *fr)
{
    if (r >= s) { *fr = 0.0; return 0.0; }
    double e2 = exp(-2.0 * a * (r - s));
    double e1 = exp(-a * (r - s));
    *fr = (r > 0.0) ? eps * (2.0 * a * e2 - 2.0 * a * e1) / r : 0.0;
    return eps * (e2 - 2.0 * e1 + 1.0);
}

/* The Mie law of Sec. II.A, U = eps [(s/r)^(2n) - 2 (s/r)^n], truncated at
 * its minimum r = s (the cut of the paper's stock code) and shifted by +eps
 * so that it is continuous there: U = eps [(s/r)^(2n) - 2 (s/r)^n + 1] for
 * r < s, 0 beyond (for n = 6 the WCA form of Lennard-Jones).  Force on i
 * from j: -dU/dr = (2n eps / r) [(s/r)^(2n) - (s/r)^n] along (x_i - x_j)/r. */
double orc_mie(double r, double s, double eps, int n, double *fr)
{
    if (r >= s) { *fr = 0.0; return 0.0; }
    double q = pow(s / r, n);
    *fr = 2.0 * n * eps * (q * q - q) / (r * r);
    return eps * (q * q - 2.0 * q + 1.0);
}

/* The pair law every routine below applies, set process-wide (default:
 * harmonic, one eps for all pairs).  kind 0 = harmonic, 1 = Morse with
 * stiffness a, 2 = Mie with exponent n = (int)a.  eps_scale = 1 gives atom i the prefactor
 * eps_i = eps sigma_i^d (Sec. II.A: prefactors scale with particle volume)
 * and a pair eps_ij = sqrt(eps_i eps_j) (the mixing rule of Sec. II.A);
 * eps_scale = 0 gives every pair eps.  Returns 0, or -1 for a bad kind. */
static int g_law_kind = 0;
static double g_law_a = 30.0;
static int g_law_eps_scale = 0;

int orc_set_law(int kind, double a, int eps_scale)
{
    if (kind < 0 || kind > 2) return -1;
    g_law_kind = kind;
    g_law_a = a;
    g_law_eps_scale = eps_scale ? 1 : 0;
    return 0;
}

/* U and |f|/r of atoms with diameters si, sj at distance r under the law
 * set above. */
static double pair_law(int d, double r, double si, double sj, double eps, double *fr)
{
    double s = 0.5 * (si + sj);
    double e = eps;
    if (g_law_eps_scale) e = sqrt((eps * pow(si, d)) * (eps * pow(sj, d)));
    if (g_law_kind == 1) return orc_morse(r, s, e, g_law_a, fr);
    if (g_law_kind == 2) return orc_mie(r, s, e, (int)g_law_a, fr);
    return orc_harmonic(r, s, e, fr);
}

/* Effective hard-sphere diameter of the Morse law, Eq. (12):
 *   sigma_eff(a, T) = integral_0^1 [1 - exp(-U_a(r)/T)] dr
 * for unit diameter and prefactor, by the midpoint rule on npts points. */
double orc_sigma_eff(double a, double T, int64_t npts)
{
    double h = 1.0 / (double)npts, sum = 0.0, fr;
    for (int64_t k = 0; k < npts; ++k) {
        double r = (k + 0.5) * h;
        sum += 1.0 - exp(-orc_morse(r, 1.0, 1.0, a, &fr) / T);
    }
    return sum * h;
}

/* Pair forces F[N*d], pair energy E = sum_{i<j} U_ij and virial
 * W = sum_{i<j} (x_i - x_j).f_ij.  With counts == NULL every pair i<j is
 * visited (brute force); otherwise counts/idx hold full Verlet lists (as
 * produced above) and each ordered pair contributes half of E and W. */
void orc_forces(int d, int64_t N, double L, const double *x, const double *sigma,
                double eps, const int32_t *counts, const int32_t *idx,
                double *F, double *E, double *W)
{
    double e = 0.0, w = 0.0;
    memset(F, 0, sizeof(double) * (size_t)(N * d));
    if (!counts) {
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t j = i + 1; j < N; ++j) {
                double dx[ORC_MAXD], r2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    dx[k] = orc_min_image(x[i * d + k] - x[j * d + k], L);
                    r2 += dx[k] * dx[k];
                }
                double fr;
                double r = sqrt(r2);
                double u = pair_law(d, r, sigma[i], sigma[j], eps, &fr);
                if (u == 0.0 && fr == 0.0) continue;
                for (int k = 0; k < d; ++k) {
                    F[i * d + k] += fr * dx[k];
                    F[j * d + k] -= fr * dx[k];
                }
                e += u;
                w += fr * r2;
            }
        }
    } else {
        int64_t *first = malloc(sizeof(int64_t) * (size_t)(N + 1));
        first[0] = 0;
        for (int64_t i = 0; i < N; ++i) first[i + 1] = first[i] + counts[i];
#pragma omp parallel for reduction(+ : e, w) schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            const int64_t off = first[i];
            for (int32_t a = 0; a < counts[i]; ++a) {
                int64_t j = idx[off + a];
                double dx[ORC_MAXD], r2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    dx[k] = orc_min_image(x[i * d + k] - x[j * d + k], L);
                    r2 += dx[k] * dx[k];
                }
                double fr;
                double r = sqrt(r2);
                double u = pair_law(d, r, sigma[i], sigma[j], eps, &fr);
                for (int k = 0; k < d; ++k) F[i * d + k] += fr * dx[k];
                e += 0.5 * u;
                w += 0.5 * fr * r2;
            }
        }
        free(first);
    }
    *E = e;
    *W = w;
}

/* Force on one atom i, F_i = sum_{j != i} f_ij over every other atom (the
 * plain definition), and i's half share of the pair energy and virial, so
 * that the shares of all atoms sum to E and W.  For sampled atoms of systems
 * too large for the all-pairs routine. */
void orc_force_on(int d, int64_t N, double L, const double *x, const double *sigma,
                  double eps, int64_t i, double *Fi, double *ei, double *wi)
{
    double e = 0.0, w = 0.0;
    for (int k = 0; k < d; ++k) Fi[k] = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (j == i) continue;
        double dx[ORC_MAXD], r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            dx[k] = orc_min_image(x[i * d + k] - x[j * d + k], L);
            r2 += dx[k] * dx[k];
        }
        double fr;
        double r = sqrt(r2);
        double u = pair_law(d, r, sigma[i], sigma[j], eps, &fr);
        for (int k = 0; k < d; ++k) Fi[k] += fr * dx[k];
        e += 0.5 * u;
        w += 0.5 * fr * r2;
    }
    *ei = e;
    *wi = w;
}

/* Kinetic energy K = (1/2) sum m v^2. */
double orc_kinetic(int d, int64_t N, const double *v, const double *mass)
{
    double k = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double m = mass ? mass[i] : 1.0, s = 0.0;
        for (int c = 0; c < d; ++c) s += v[i * d + c] * v[i * d + c];
        k += 0.5 * m * s;
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* neighbor-list bookkeeping shared by the MD and FIRE loops            */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t *counts, *idx;
    int64_t cap;
    double *x0;      /* positions at the last build */
    int64_t builds;
} orc_vl;

/* Build the list the way the paper does: linked subcells when
 * n_cell > 3, the all-pairs routine otherwise (Sec. II.C, last paragraph). */
static void vl_build(orc_vl *vl, int d, int64_t N, double L, const double *x,
                     const double *sigma, double skin)
{
    double smax = max_of(sigma, N);
    int n = orc_n_cell(L, smax + skin);
    int64_t (*fn)(int, int64_t, double, const double *, const double *, double, int,
                  int32_t *, int32_t *, int64_t) =
        n > 3 ? orc_neighbors_cells : orc_neighbors_brute;
    if (!vl->counts) vl->counts = malloc(sizeof(int32_t) * (size_t)N);
    if (!vl->idx) {
        vl->cap = 64 * N + 16;
        vl->idx = malloc(sizeof(int32_t) * (size_t)vl->cap);
    }
    while (fn(d, N, L, x, sigma, skin, 0, vl->counts, vl->idx, vl->cap) < 0) {
        vl->cap *= 2;
        vl->idx = realloc(vl->idx, sizeof(int32_t) * (size_t)vl->cap);
    }
    if (!vl->x0) vl->x0 = malloc(sizeof(double) * (size_t)(N * d));
    memcpy(vl->x0, x, sizeof(double) * (size_t)(N * d));
    vl->builds++;
}

/* Rebuild trigger.  Reading of Sec. II.C: the paper's rule (0.1 % of atoms
 * moved s/2, or any atom moved s) can miss a pair closing from both sides,
 * so the oracle rebuilds as soon as 2 max_i |x_i - x_i(build)| > skin, which
 * keeps every list exact. */
static int vl_needs_rebuild(const orc_vl *vl, int d, int64_t N, double L,
                            const double *x, double skin)
{
    double dmax2 = 0.0;
#pragma omp parallel for reduction(max : dmax2) schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double dx = orc_min_image(x[i * d + k] - vl->x0[i * d + k], L);
            s += dx * dx;
        }
        if (s > dmax2) dmax2 = s;
    }
    return 4.0 * dmax2 > skin * skin;
}

/* The paper's rule (Sec. II.C): rebuild when at least 0.1 % of the atoms
 * have moved by at least s/2, or any atom by at least s, since the build.
 * Unlike the rule above it can miss a pair that closes from both sides. */
static int vl_needs_rebuild_paper(const orc_vl *vl, int d, int64_t N, double L,
                                  const double *x, double skin)
{
    int64_t half = 0;
    int any = 0;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
            double dx = orc_min_image(x[i * d + k] - vl->x0[i * d + k], L);
            s += dx * dx;
        }
        if (s >= 0.25 * skin * skin) half++;
        if (s >= skin * skin) any = 1;
    }
    return any || (double)half >= 0.001 * (double)N;
}

static void vl_free(orc_vl *vl)
{
    free(vl->counts); free(vl->idx); free(vl->x0);
}

/* Wrap one coordinate back into [-L/2, L/2), counting box crossings. */
static double wrap(double x, double L, int32_t *img)
{
    if (x >= 0.5 * L) { x -= L; if (img) ++*img; }
    else if (x < -0.5 * L) { x += L; if (img) --*img; }
    return x;
}

/* ------------------------------------------------------------------ */
/* velocity Verlet                                                      */
/* ------------------------------------------------------------------ */

/* nsteps of kick-drift-kick velocity Verlet (Sec. II.B: the leapfrog
 * "kick-drift-kick" variant).  One step:
 *   v += (dt/2) F/m;  x += dt v, wrapped with image counts;
 *   rebuild the Verlet list if the trigger fires;  F = F(x);
 *   v += (dt/2) F/m;
 *   with tau > 0 (NVT): v *= lambda, the Berendsen factor (Berendsen et al.
 *   1984, the thermostat of Sec. II.E, applied in the second kick as the
 *   paper does) lambda = sqrt(1 + (dt/tau)(T_target/T - 1)), where T is the
 *   kinetic temperature 2K/(d(N-1)) at the end of the previous step (at the
 *   start of the call for the first step), and lambda = 1 when T = 0.
 * rule 0 rebuilds the list when 2 max|dx| > s after any drift (exact
 * forces); rule 1 applies the paper's rule (vl_needs_rebuild_paper) after
 * every n_bet-th step, *step_count counting the steps across calls.
 * F must hold the forces at the incoming x (have_F != 0) or is computed
 * first from the list (have_F == 0); it holds those at the outgoing x on
 * return.  thermo[0..2] = E_pair, virial W, kinetic K at the end.
 * Returns the number of list builds (the first one included). */
int64_t orc_md_steps(int d, int64_t N, double L, double *x, double *v, int32_t *img,
                     const double *sigma, const double *mass, double eps,
                     double skin, double dt, int64_t nsteps, double *F, int have_F,
                     double *thermo, double T_target, double tau, int rule, int64_t n_bet,
                     int64_t *step_count)
{
    orc_vl vl = {0};
    double E = 0.0, W = 0.0;
    double T_prev = 2.0 * orc_kinetic(d, N, v, mass) / ((double)d * (double)(N - 1));
    vl_build(&vl, d, N, L, x, sigma, skin);
    if (!have_F) orc_forces(d, N, L, x, sigma, eps, vl.counts, vl.idx, F, &E, &W);
    for (int64_t step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double m = mass ? mass[i] : 1.0;
            for (int k = 0; k < d; ++k) {
                v[i * d + k] += 0.5 * dt * F[i * d + k] / m;
                x[i * d + k] += dt * v[i * d + k];
                x[i * d + k] = wrap(x[i * d + k], L, img ? &img[i * d + k] : NULL);
            }
        }
        if (rule == 1) {   /* the paper's rule, checked every n_bet steps */
            *step_count += 1;
            if (*step_count % n_bet == 0 && vl_needs_rebuild_paper(&vl, d, N, L, x, skin))
                vl_build(&vl, d, N, L, x, sigma, skin);
        } else if (vl_needs_rebuild(&vl, d, N, L, x, skin)) {
            vl_build(&vl, d, N, L, x, sigma, skin);
        }
        orc_forces(d, N, L, x, sigma, eps, vl.counts, vl.idx, F, &E, &W);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double m = mass ? mass[i] : 1.0;
            for (int k = 0; k < d; ++k) v[i * d + k] += 0.5 * dt * F[i * d + k] / m;
        }
        if (tau > 0.0) {
            double lambda = 1.0;
            if (T_prev > 0.0) lambda = sqrt(fmax(0.0, 1.0 + (dt / tau) * (T_target / T_prev - 1.0)));
            for (int64_t a = 0; a < N * d; ++a) v[a] *= lambda;
            T_prev = 2.0 * orc_kinetic(d, N, v, mass) / ((double)d * (double)(N - 1));
        }
    }
    if (nsteps == 0) orc_forces(d, N, L, x, sigma, eps, vl.counts, vl.idx, F, &E, &W);
    thermo[0] = E;
    thermo[1] = W;
    thermo[2] = orc_kinetic(d, N, v, mass);
    int64_t b = vl.builds;
    vl_free(&vl);
    return b;
}

/* ------------------------------------------------------------------ */
/* FIRE 2.0                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    double dt0, dt_max, dt_min, f_inc, f_dec, alpha0, f_alpha, f_tol;
    int64_t n_delay, n_neg_max, max_iter;
    int initial_delay;
    double e_thres, f_thres, dx_max;   /* the paper's options; 0 = off */
} orc_fire_params;

/* FIRE 2.0 energy minimisation with the semi-implicit Euler integrator
 * (Sec. II.B; Guenole et al., Comput. Mater. Sci. 175, 109584 (2020)).
 * The paper cites the method and prints no step, so the steps below are
 * the published algorithm, in order, with these readings:
 *   - stop when max_i |F_i| < f_tol (per-atom Euclidean norm), tested before
 *     each iteration; or after max_iter iterations; or after more than
 *     n_neg_max consecutive P <= 0 steps;
 *   - P = F.v over all atoms; on P > 0: Npos += 1, Nneg = 0, and after
 *     n_delay such steps dt = min(f_inc dt, dt_max), alpha *= f_alpha;
 *     on P <= 0: Npos = 0, Nneg += 1; unless still inside the initial
 *     delay, dt is multiplied by f_dec only when f_dec dt >= dt_min (it is
 *     left as it is otherwise) and alpha = alpha0; then x -= (dt/2) v and
 *     v = 0;
 *   - the MD integration step, the same on both branches: v += dt F/m;
 *     v = (1-alpha) v + alpha |v| F/|F| with norms over all atoms (after a
 *     P <= 0 step v = dt F/m, which the mixing leaves alone only when all
 *     masses are equal); x += dt v; F = F(x).
 * The paper's own stop criteria (Sec. II.B), each off when 0: the average
 * pair energy E_pair/N below e_thres; or the fractional energy drop
 * |(E_{i+1} - E_i)/E_i| (Eq. (6)) below f_thres for ten consecutive
 * iterations.  dx_max > 0 (Table II's maximum displacement per time step):
 * an atom whose move (the step dt v_i, or the back-off (dt/2) v_i) is
 * longer than dx_max moves dx_max along it instead.
 * v is zeroed on entry.  out[0..3] = iterations, final E_pair, final
 * max_i |F_i|, builds.  Returns 0 on convergence, 1 if max_iter was hit,
 * 2 if the P <= 0 count ran out. */
int orc_fire(int d, int64_t N, double L, double *x, double *v, int32_t *img,
             const double *sigma, const double *mass, double eps, double skin,
             const orc_fire_params *p, double *F, double *out)
{
    orc_vl vl = {0};
    double E = 0.0, W = 0.0, dt = p->dt0, alpha = p->alpha0;
    int64_t npos = 0, nneg = 0, it = 0;
    int status = 1;
    memset(v, 0, sizeof(double) * (size_t)(N * d));
    vl_build(&vl, d, N, L, x, sigma, skin);
    orc_forces(d, N, L, x, sigma, eps, vl.counts, vl.idx, F, &E, &W);
    double E_prev = 0.0;
    int64_t nflat = 0;
    for (;;) {
        double fmax2 = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += F[i * d + k] * F[i * d + k];
            if (s > fmax2) fmax2 = s;
        }
        if (p->f_thres > 0.0) {
            if (it > 0 && E_prev != 0.0 && fabs((E - E_prev) / E_prev) < p->f_thres) nflat++;
            else nflat = 0;
            E_prev = E;
        }
        if (sqrt(fmax2) < p->f_tol) { status = 0; break; }
        if (p->e_thres > 0.0 && E / (double)N < p->e_thres) { status = 0; break; }
        if (p->f_thres > 0.0 && nflat >= 10) { status = 0; break; }
        if (it >= p->max_iter) { status = 1; break; }

        double P = 0.0;
        for (int64_t a = 0; a < N * d; ++a) P += F[a] * v[a];
        if (P > 0.0) {
            npos++;
            nneg = 0;
            if (npos > p->n_delay) {
                dt = fmin(dt * p->f_inc, p->dt_max);
                alpha *= p->f_alpha;
            }
        } else {
            npos = 0;
            nneg++;
            if (nneg > p->n_neg_max) { status = 2; break; }
            if (!(p->initial_delay && it < p->n_delay)) {
                if (dt * p->f_dec >= p->dt_min) dt *= p->f_dec;
                alpha = p->alpha0;
            }
            for (int64_t i = 0; i < N; ++i) {
                double c = 1.0;
                if (p->dx_max > 0.0) {
                    double st2 = 0.0;
                    for (int k = 0; k < d; ++k) st2 += (0.5 * dt * v[i * d + k]) * (0.5 * dt * v[i * d + k]);
                    if (st2 > p->dx_max * p->dx_max) c = p->dx_max / sqrt(st2);
                }
                for (int k = 0; k < d; ++k) {
                    x[i * d + k] -= c * (0.5 * dt * v[i * d + k]);
                    v[i * d + k] = 0.0;
                }
            }
        }
        for (int64_t i = 0; i < N; ++i) {
            double m = mass ? mass[i] : 1.0;
            for (int k = 0; k < d; ++k) v[i * d + k] += dt * F[i * d + k] / m;
        }
        {
            double vv = 0.0, ff = 0.0;
            for (int64_t a = 0; a < N * d; ++a) { vv += v[a] * v[a]; ff += F[a] * F[a]; }
            double vn = sqrt(vv), fn = sqrt(ff);
            if (fn > 0.0)
                for (int64_t a = 0; a < N * d; ++a)
                    v[a] = (1.0 - alpha) * v[a] + alpha * vn * F[a] / fn;
        }
        for (int64_t i = 0; i < N; ++i) {
            double c = 1.0;
            if (p->dx_max > 0.0) {
                double st2 = 0.0;
                for (int k = 0; k < d; ++k) st2 += (dt * v[i * d + k]) * (dt * v[i * d + k]);
                if (st2 > p->dx_max * p->dx_max) c = p->dx_max / sqrt(st2);
            }
            for (int k = 0; k < d; ++k) {
                x[i * d + k] += c * (dt * v[i * d + k]);
                x[i * d + k] = wrap(x[i * d + k], L, img ? &img[i * d + k] : NULL);
            }
        }
        if (vl_needs_rebuild(&vl, d, N, L, x, skin)) vl_build(&vl, d, N, L, x, sigma, skin);
        orc_forces(d, N, L, x, sigma, eps, vl.counts, vl.idx, F, &E, &W);
        it++;
    }
    double fmax2 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += F[i * d + k] * F[i * d + k];
        if (s > fmax2) fmax2 = s;
    }
    out[0] = (double)it;
    out[1] = E;
    out[2] = sqrt(fmax2);
    out[3] = (double)vl.builds;
    vl_free(&vl);
    return status;
}

/* NPT with the Berendsen barostat (Berendsen et al. 1984; Sec. II.E):
 * nsteps of orc_md_steps (NVE, or NVT when tau > 0) in pieces of n_baro
 * steps; after each full piece the pressure P = (2K + W)/(d L^d) of its end
 * state gives mu = [1 - beta (n_baro dt / tau_P)(P_target - P)]^(1/d), and
 * every position and the box side are multiplied by mu (the box stays
 * centred at the origin).  *count carries the steps since the last rescale
 * across calls.  *L is updated.  thermo as orc_md_steps, for the end state
 * (after a final rescale, at the rescaled positions).  Returns the number of
 * rescales, or -1 if one would make the box vanish. */
int64_t orc_md_npt(int d, int64_t N, double *L, double *x, double *v, int32_t *img,
                   const double *sigma, const double *mass, double eps, double skin,
                   double dt, int64_t nsteps, double T_target, double tau,
                   double P_target, double tau_P, double beta, int64_t n_baro,
                   int64_t *count, double *thermo)
{
    double *F = (double *)malloc(sizeof(double) * (size_t)(N * d));
    int64_t left = nsteps, nresc = 0;
    int rescaled_last = 0;
    thermo[0] = thermo[1] = thermo[2] = 0.0;
    while (left > 0) {
        int64_t chunk = n_baro - *count;
        if (chunk > left) chunk = left;
        int64_t st0 = 0;
        orc_md_steps(d, N, *L, x, v, img, sigma, mass, eps, skin, dt, chunk, F, 0, thermo,
                     T_target, tau, 0, 1, &st0);
        left -= chunk;
        *count += chunk;
        rescaled_last = 0;
        if (*count == n_baro) {
            double V = pow(*L, d);
            double P = (2.0 * thermo[2] + thermo[1]) / (d * V);
            double base = 1.0 - beta * ((double)n_baro * dt / tau_P) * (P_target - P);
            if (!(base > 0.0)) { free(F); return -1; }
            double mu = pow(base, 1.0 / d);
            for (int64_t a = 0; a < N * d; ++a) x[a] *= mu;
            *L *= mu;
            *count = 0;
            ++nresc;
            rescaled_last = 1;
        }
    }
    if (rescaled_last) {
        int64_t st0 = 0;
        orc_md_steps(d, N, *L, x, v, img, sigma, mass, eps, skin, dt, 0, F, 0, thermo, T_target,
                     tau, 0, 1, &st0);
    }
    free(F);
    return nresc;
}

/* ------------------------------------------------------------------ */
/* observables (Sec. II.E)                                              */
/* ------------------------------------------------------------------ */

/* Against the reference configuration xref (both unwrapped, row-major):
 *   out[0] = <|dr|^2>, out[1] = <|dr|^4>,
 *   out[2] = alpha_2 = d <|dr|^4> / ((d + 2) <|dr|^2>^2) - 1  (Eq. (14)),
 *   out[3] = f_ov = (1/N) sum_i Theta(a - |dr_i|), Theta(0) = 0 (Eq. (15)),
 *   out[4] = Z = (1/N) sum_i #{j != i : r_ij < sigma_ij} at positions x
 *            (minimum image), by brute force over all pairs (0 when sigma
 *            is NULL);
 * gs[b] (nbins > 0) = (1/N) sum_i [b w <= |dr_i| < (b+1) w] / w, w = r_max /
 * nbins: the self part of the van Hove function (Eq. (16)) with its delta
 * function smeared over bins of width w. */
void orc_observables(int d, int64_t N, double L, const double *x, const double *xref,
                     const double *sigma, double a, int nbins, double r_max,
                     double *out, double *gs)
{
    double s2 = 0.0, s4 = 0.0, nov = 0.0, nz = 0.0;
    double w = nbins > 0 ? r_max / nbins : 1.0;
    for (int b = 0; b < nbins; ++b) gs[b] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double r2 = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = x[i * d + k] - xref[i * d + k];
            r2 += t * t;
        }
        s2 += r2;
        s4 += r2 * r2;
        double r = sqrt(r2);
        if (r < a) nov += 1.0;
        if (nbins > 0 && r < r_max) {
            int b = (int)floor(r / w);
            if (b < nbins) gs[b] += 1.0;
        }
        for (int64_t j = 0; sigma && j < N; ++j) {
            if (j == i) continue;
            double sij = 0.5 * (sigma[i] + sigma[j]);
            if (dist2(d, L, x, i, j) < sij * sij) nz += 1.0;
        }
    }
    for (int b = 0; b < nbins; ++b) gs[b] /= (double)N * w;
    out[0] = s2 / N;
    out[1] = s4 / N;
    out[2] = out[0] > 0.0 ? d * out[1] / ((d + 2.0) * out[0] * out[0]) - 1.0 : 0.0;
    out[3] = nov / N;
    out[4] = nz / N;
}

/* ------------------------------------------------------------------ */
/* SWAP Monte Carlo                                                     */
/* ------------------------------------------------------------------ */

/* Interaction energy of atom a, given the diameter sa, with every atom
 * except a and b (the swap partner), by brute force over all atoms. */
static double energy_with(int d, int64_t N, double L, const double *x,
                          const double *sigma, double eps, int64_t a, double sa,
                          int64_t b)
{
    double e = 0.0, fr;
    for (int64_t k = 0; k < N; ++k) {
        if (k == a || k == b) continue;
        double r = sqrt(dist2(d, L, x, a, k));
        e += pair_law(d, r, sa, sigma[k], eps, &fr);
    }
    return e;
}

/* One SWAP pass over npairs candidate pairs, serially and in order
 * (Sec. II.D).  For pair (i, j): E_b (Eq. (10)) and E_a (Eq. (11)) are the
 * energies of i and j with all other atoms before and after exchanging
 * their diameters.  Reading: the partner is excluded from both sums (the
 * i-j term is unchanged by the exchange).  Metropolis: accept iff
 * u < exp(-(E_a - E_b)/T).  On acceptance sigma and mass are exchanged and
 * each velocity is rescaled by sqrt(m_old/m_new) so that each atom keeps
 * its kinetic energy.  accepted[k] (nullable) records each decision.
 * Returns the number of accepted exchanges. */
int64_t orc_swap(int d, int64_t N, double L, const double *x, double *sigma,
                 double *mass, double *v, double eps, double T, int64_t npairs,
                 const int32_t *pairs, const double *uniforms, int8_t *accepted)
{
    int64_t nacc = 0;
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t i = pairs[2 * p], j = pairs[2 * p + 1];
        int acc = 0;
        if (i != j) {
            double Eb = energy_with(d, N, L, x, sigma, eps, i, sigma[i], j)
                      + energy_with(d, N, L, x, sigma, eps, j, sigma[j], i);
            double Ea = energy_with(d, N, L, x, sigma, eps, i, sigma[j], j)
                      + energy_with(d, N, L, x, sigma, eps, j, sigma[i], i);
            acc = uniforms[p] < exp(-(Ea - Eb) / T);
        }
        if (acc) {
            double t = sigma[i]; sigma[i] = sigma[j]; sigma[j] = t;
            if (mass) {
                double mi = mass[i], mj = mass[j];
                if (v) {
                    for (int k = 0; k < d; ++k) {
                        v[i * d + k] *= sqrt(mi / mj);
                        v[j * d + k] *= sqrt(mj / mi);
                    }
                }
                mass[i] = mj; mass[j] = mi;
            }
            ++nacc;
        }
        if (accepted) accepted[p] = (int8_t)acc;
    }
    return nacc;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 and the seeded SWAP draw                               */
/* ------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds, from its published definition (Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
 * each round multiplies words 0 and 2 by two fixed odd constants, mixes the
 * high halves with words 1 and 3 and the key, and the key is advanced by
 * two Weyl increments between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Candidate pair p of SWAP pass `sweep` under `seed`: one Philox block at
 * counter (p, sweep, 0x53574150, 0) and key (seed low, seed high) gives
 * i = floor(w0 N / 2^32), j' = floor(w1 (N-1) / 2^32), j = j' + (j' >= i)
 * (so j != i, both uniform), and u = (w2 + 2^32 w3) / 2^64 truncated to
 * 53 bits, in [0, 1). */
void orc_swap_draw(uint64_t seed, int64_t sweep, int64_t npairs, int64_t N,
                   int32_t *pairs, double *uniforms)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t p = 0; p < npairs; ++p) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)sweep, 0x53574150u, 0u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        int64_t i = (int64_t)(((uint64_t)w[0] * (uint64_t)N) >> 32);
        int64_t j = (int64_t)(((uint64_t)w[1] * (uint64_t)(N - 1)) >> 32);
        if (j >= i) ++j;
        uint64_t bits = ((uint64_t)w[3] << 32) | w[2];
        pairs[2 * p] = (int32_t)i;
        pairs[2 * p + 1] = (int32_t)j;
        uniforms[p] = (double)(bits >> 11) * (1.0 / 9007199254740992.0);
    }
}
