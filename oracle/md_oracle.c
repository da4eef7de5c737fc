/*
 * md_oracle.c -- plain, slow, FP64 CPU reference for the soft-sphere
 * molecular-dynamics step of Rapaport, "Enhanced molecular dynamics
 * performance with a programmable graphics processor" (arXiv 0911.5631).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline arm may load this library.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is double precision, compiled without FP contraction
 * (-ffp-contract=off), in the order the paper states.  The parity reference
 * is the plain single-threaded build.  The same source compiled with
 * -fopenmp gives the threaded build that only times the oracle on all host
 * cores: the cell loop of the pair enumeration and the pair loop of the
 * forces are cut into as many contiguous chunks as there are threads, and
 * the chunks' results are joined in chunk order (pair lists concatenated,
 * force arrays and sums added chunk by chunk), so with one chunk both builds
 * are the same program and with several the pair list is the same list and
 * only the order of the force sums differs.
 *
 *
 *   - pair potential: Eq. (1) (Lennard-Jones) truncated at r_c, plus a
 *     constant shift; the soft-sphere (SP, WCA) case is r_c = 2^(1/6) with a
 *     shift of +epsilon (Sec. 3.1).  Reduced units sigma = epsilon = m = 1.
 *   - region: centred at the origin, edge L_d, cell grid G_d = floor(L_d/r_n),
 *     cell width w_d = L_d/G_d (Sec. 3.1); optional rounding of G_d down to
 *     an even number, which is what every cell count printed in Tables 1
 *     and 5 corresponds to.
 *   - cell assignment by linked lists and the half-shell (14 offsets) pair
 *     enumeration with periodic-image shifts beta (Sec. 3.2).
 *   - pair-list force evaluation using Newton's third law (Sec. 3.2).
 *   - the step loop (a)-(f) of Sec. 3.1: half kick + drift; periodic wrap
 *     and rebuild when the largest displacement since the last rebuild
 *     reaches delta/2; forces; half kick; properties; optional velocity
 *     rescaling during equilibration.
 *
 * Brute-force O(N^2) minimum-image versions of the pair enumeration and of
 * the forces are included; the tests use them to pin the cell-list code.
 *
 * Function names carry the prefix "orc_".  Positions and velocities are
 * N x 3 row-major (x, y, z per atom).  Pairs are int32 (i, j) with i < j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of chunks the two big loops are cut into: the threads of the
 * threaded build, 1 otherwise. */
static int n_chunks(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of threads the oracle runs on (1 in the plain build). */
int orc_threads(void)
{
    return n_chunks();
}

/* ------------------------------------------------------------------ */
/* Pair term                                                           */
/* ------------------------------------------------------------------ */

/* Eq. (1) with sigma = epsilon = 1, written in terms of r^2.  Returns
 * u(r) + ushift in *u and the scalar fr such that the force on atom i from
 * atom j is fr * (r_i - r_j), i.e. fr = -(du/dr)/r = 48 r^-14 - 24 r^-8. */
void orc_pair(double r2, double ushift, double* fr, double* u)
{
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    *u = 4.0 * ir6 * (ir6 - 1.0) + ushift;
    *fr = 48.0 * ir6 * (ir6 - 0.5) * ir2;
}

/* ------------------------------------------------------------------ */
/* Region and cells (Sec. 3.1, Sec. 3.2)                               */
/* ------------------------------------------------------------------ */

/* G_d = floor(L_d / r_n); with even != 0 rounded down to an even count.
 * Returns 0, or -1 if some G_d < 3 (the 27-cell neighbourhood would then
 * visit one cell twice). */
int orc_cell_grid(const double L[3], double rn, int even, int G[3])
{
    int ok = 0;
    for (int d = 0; d < 3; d++) {
        int g = (int)floor(L[d] / rn);
        if (even) g -= g % 2;
        G[d] = g;
        if (g < 3) ok = -1;
    }
    return ok;
}

/* Periodic wrap into [-L/2, L/2): x <- x - L floor((x + L/2) / L), the
 * division written as a product with 1/L. */
void orc_wrap(int64_t n, double* pos, const double L[3])
{
    for (int d = 0; d < 3; d++) {
        double hL = 0.5 * L[d];
        double invL = 1.0 / L[d];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double x = pos[3 * i + d];
            double s = floor((x + hL) * invL);
            pos[3 * i + d] = x - s * L[d];
        }
    }
}

/* Component cell coordinate: shift the centred region to [0, L), scale by
 * G/L and truncate; an atom at the upper face (only possible through
 * rounding) goes to cell 0 and one below the lower face to cell G-1. */
static int cell_coord(double x, double hL, double invW, int G)
{
    int c = (int)floor((x + hL) * invW);
    if (c >= G) c -= G;
    if (c < 0) c += G;
    return c;
}

/* Scalar cell index, 0-based form of the paper's
 * c = ((c_z - 1) G_y + c_y - 1) G_x + c_x. */
void orc_cell_of(int64_t n, const double* pos, const double L[3], const int G[3], int32_t* cell)
{
    double hL[3], invW[3];
    for (int d = 0; d < 3; d++) {
        hL[d] = 0.5 * L[d];
        invW[d] = (double)G[d] / L[d];
    }
    for (int64_t i = 0; i < n; i++) {
        int cx = cell_coord(pos[3 * i + 0], hL[0], invW[0], G[0]);
        int cy = cell_coord(pos[3 * i + 1], hL[1], invW[1], G[1]);
        int cz = cell_coord(pos[3 * i + 2], hL[2], invW[2], G[2]);
        cell[i] = (int32_t)((cz * G[1] + cy) * G[0] + cx);
    }
}

/* ------------------------------------------------------------------ */
/* Pair lists                                                          */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t i, j;          /* atoms, any order */
    int8_t s[3];           /* periodic shift b = s * L, added to r_i - r_j */
} pair_t;

typedef struct {
    pair_t* p;
    int64_t n, cap;
} pairlist_t;

static int pl_push(pairlist_t* pl, int32_t i, int32_t j, const int s[3])
{
    if (pl->n == pl->cap) {
        int64_t nc = pl->cap ? 2 * pl->cap : 1024;
        pair_t* q = (pair_t*)realloc(pl->p, (size_t)nc * sizeof(pair_t));
        if (!q) return -1;
        pl->p = q;
        pl->cap = nc;
    }
    pair_t* e = &pl->p[pl->n++];
    e->i = i;
    e->j = j;
    e->s[0] = (int8_t)s[0];
    e->s[1] = (int8_t)s[1];
    e->s[2] = (int8_t)s[2];
    return 0;
}

/* The 14 cell offsets of the half shell: the cell itself and 13 of its 26
 * neighbours, one from each +/- pair (Sec. 3.2). */
static const int HALF_SHELL[14][3] = {
    {0, 0, 0},  {1, 0, 0},  {1, 1, 0},  {0, 1, 0},  {-1, 1, 0},
    {0, 0, 1},  {1, 0, 1},  {1, 1, 1},  {0, 1, 1},  {-1, 1, 1},
    {-1, 0, 1}, {-1, -1, 1}, {0, -1, 1}, {1, -1, 1}};

/* The pairs of the cells c1 in [c_beg, c_end) with the cells of their half
 * shell, given the linked lists head/next (Sec. 3.2).  Each pair with
 * |r_i - r_j + b| < rcut is recorded once together with its shift b. */
static int pairs_of_cells(const double* pos, const double L[3], const int G[3], const int32_t* head,
                          const int32_t* next, double rcut, int64_t c_beg, int64_t c_end, pairlist_t* pl)
{
    double rc2 = rcut * rcut;
    for (int64_t c1 = c_beg; c1 < c_end; c1++) {
        int cx = (int)(c1 % G[0]), cy = (int)((c1 / G[0]) % G[1]), cz = (int)(c1 / ((int64_t)G[0] * G[1]));
        for (int k = 0; k < 14; k++) {
            int cc[3] = {cx + HALF_SHELL[k][0], cy + HALF_SHELL[k][1], cz + HALF_SHELL[k][2]};
            int s[3];
            /* A neighbour cell across the upper face holds atoms near the
             * lower face: their image near c1 is r + L, so b = -L.  Across
             * the lower face the opposite. */
            for (int d = 0; d < 3; d++) {
                s[d] = 0;
                if (cc[d] >= G[d]) { cc[d] -= G[d]; s[d] = -1; }
                else if (cc[d] < 0) { cc[d] += G[d]; s[d] = 1; }
            }
            int32_t c2 = (cc[2] * G[1] + cc[1]) * G[0] + cc[0];
            for (int32_t i1 = head[c1]; i1 >= 0; i1 = next[i1]) {
                for (int32_t i2 = head[c2]; i2 >= 0; i2 = next[i2]) {
                    if (c1 == c2 && !(i1 < i2)) continue;
                    double dx = pos[3 * i1 + 0] - pos[3 * i2 + 0] + s[0] * L[0];
                    double dy = pos[3 * i1 + 1] - pos[3 * i2 + 1] + s[1] * L[1];
                    double dz = pos[3 * i1 + 2] - pos[3 * i2 + 2] + s[2] * L[2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rc2) {
                        if (pl_push(pl, i1, i2, s)) return -1;
                    }
                }
            }
        }
    }
    return 0;
}

/* Linked-list cell assignment and half-shell pair enumeration with cutoff
 * rcut (Sec. 3.2), cells taken in the order c = (c_z G_y + c_y) G_x + c_x.
 * Positions must lie in [-L/2, L/2).  The cell range is cut into n_chunks()
 * contiguous pieces whose lists are concatenated in order, which is the
 * list one pass over all cells makes. */
static int build_pairs_cells(int64_t n, const double* pos, const double L[3], const int G[3],
                             double rcut, pairlist_t* pl)
{
    int64_t nc = (int64_t)G[0] * G[1] * G[2];
    int32_t* head = (int32_t*)malloc((size_t)nc * sizeof(int32_t));
    int32_t* next = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* cell = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int nch = n_chunks();
    pairlist_t* part = (pairlist_t*)calloc((size_t)nch, sizeof(pairlist_t));
    if (!head || !next || !cell || !part) {
        free(head); free(next); free(cell); free(part);
        return -1;
    }
    for (int64_t c = 0; c < nc; c++) head[c] = -1;
    orc_cell_of(n, pos, L, G, cell);
    for (int64_t i = 0; i < n; i++) {
        next[i] = head[cell[i]];
        head[cell[i]] = (int32_t)i;
    }
    int err = 0;
    if (nch == 1) {
        pl->n = 0;
        err = pairs_of_cells(pos, L, G, head, next, rcut, 0, nc, pl);
    } else {
#pragma omp parallel for schedule(static, 1) reduction(| : err)
        for (int k = 0; k < nch; k++)
            err |= pairs_of_cells(pos, L, G, head, next, rcut, nc * k / nch, nc * (k + 1) / nch, &part[k]);
        int64_t total = 0;
        for (int k = 0; k < nch; k++) total += part[k].n;
        if (!err && total > pl->cap) {
            pair_t* q = (pair_t*)realloc(pl->p, (size_t)(total > 0 ? total : 1) * sizeof(pair_t));
            if (q) { pl->p = q; pl->cap = total; }
            else err = 1;
        }
        pl->n = 0;
        for (int k = 0; k < nch && !err; k++) {
            if (part[k].n) memcpy(pl->p + pl->n, part[k].p, (size_t)part[k].n * sizeof(pair_t));
            pl->n += part[k].n;
        }
        for (int k = 0; k < nch; k++) free(part[k].p);
    }
    free(head); free(next); free(cell); free(part);
    return err ? -1 : 0;
}

static void emit_pairs(const pairlist_t* pl, int64_t cap, int32_t* out)
{
    for (int64_t m = 0; m < pl->n && m < cap; m++) {
        int32_t a = pl->p[m].i, b = pl->p[m].j;
        out[2 * m + 0] = a < b ? a : b;
        out[2 * m + 1] = a < b ? b : a;
    }
}

/* All pairs within rcut through the cell lists.  Writes up to cap pairs
 * (i < j) and returns the total count, or -1 on bad geometry / memory. */
int64_t orc_pairs_cells(int64_t n, const double* pos, const double L[3], const int G[3],
                        double rcut, int64_t cap, int32_t* pairs)
{
    if (G[0] < 3 || G[1] < 3 || G[2] < 3) return -1;
    pairlist_t pl = {0, 0, 0};
    if (build_pairs_cells(n, pos, L, G, rcut, &pl)) { free(pl.p); return -1; }
    emit_pairs(&pl, cap, pairs);
    int64_t np = pl.n;
    free(pl.p);
    return np;
}

/* Minimum-image separation component. */
static double min_image(double dx, double Ld)
{
    return dx - Ld * round(dx / Ld);
}

/* All pairs within rcut by direct O(N^2) enumeration with the minimum-image
 * convention; the definition the cell lists must reproduce. */
int64_t orc_pairs_brute(int64_t n, const double* pos, const double L[3], double rcut,
                        int64_t cap, int32_t* pairs)
{
    double rc2 = rcut * rcut;
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], L[0]);
            double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L[1]);
            double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L[2]);
            if (dx * dx + dy * dy + dz * dz < rc2) {
                if (m < cap) {
                    pairs[2 * m + 0] = (int32_t)i;
                    pairs[2 * m + 1] = (int32_t)j;
                }
                m++;
            }
        }
    return m;
}

/* Minimum-image squared distance of one pair (for classifying pairs that lie
 * within rounding of a cutoff). */
double orc_pair_r2(const double* pos, const double L[3], int64_t i, int64_t j)
{
    double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], L[0]);
    double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L[1]);
    double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L[2]);
    return dx * dx + dy * dy + dz * dz;
}

/* ------------------------------------------------------------------ */
/* Forces, energy, virial                                              */
/* ------------------------------------------------------------------ */

/* The pairs [m_beg, m_end) of a pair list: each pair within rc adds fr * r
 * to atom i and subtracts it from atom j in f (Newton's third law,
 * Sec. 3.2); U and W, the sums of u(r) and r . f, are added to *pe, *vir. */
static void forces_of_pairs(const double* pos, const double L[3], const pairlist_t* pl, int64_t m_beg,
                            int64_t m_end, double rc, double ushift, double* f, double* pe, double* vir)
{
    double rc2 = rc * rc;
    double U = 0.0, W = 0.0;
    for (int64_t m = m_beg; m < m_end; m++) {
        const pair_t* e = &pl->p[m];
        double dx = pos[3 * e->i + 0] - pos[3 * e->j + 0] + e->s[0] * L[0];
        double dy = pos[3 * e->i + 1] - pos[3 * e->j + 1] + e->s[1] * L[1];
        double dz = pos[3 * e->i + 2] - pos[3 * e->j + 2] + e->s[2] * L[2];
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
            double fr, u;
            orc_pair(r2, ushift, &fr, &u);
            f[3 * e->i + 0] += fr * dx;
            f[3 * e->i + 1] += fr * dy;
            f[3 * e->i + 2] += fr * dz;
            f[3 * e->j + 0] -= fr * dx;
            f[3 * e->j + 1] -= fr * dy;
            f[3 * e->j + 2] -= fr * dz;
            U += u;
            W += fr * r2;
        }
    }
    *pe = U;
    *vir = W;
}

/* Force arrays of the chunks k > 0 (none with a single chunk). */
static double* chunk_forces_alloc(int64_t n)
{
    int nch = n_chunks();
    if (nch == 1) return NULL;
    return (double*)malloc((size_t)(nch - 1) * (size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
}

/* Pair-list force evaluation (forces_of_pairs over the whole list).  With
 * several chunks, chunk k > 0 sums into its own array of fk, and the arrays
 * and the chunk sums are added in chunk order afterwards. */
static void forces_from_pairs(int64_t n, const double* pos, const double L[3], const pairlist_t* pl,
                              double rc, double ushift, double* f, double* fk, double* pe, double* vir)
{
    int nch = n_chunks();
    if (nch == 1 || !fk) {
        memset(f, 0, (size_t)n * 3 * sizeof(double));
        forces_of_pairs(pos, L, pl, 0, pl->n, rc, ushift, f, pe, vir);
        return;
    }
    double sums[2 * 1024];
    if (nch > 1024) nch = 1024;
#pragma omp parallel for schedule(static, 1)
    for (int k = 0; k < nch; k++) {
        double* fo = k == 0 ? f : fk + (size_t)(k - 1) * (size_t)n * 3;
        memset(fo, 0, (size_t)n * 3 * sizeof(double));
        forces_of_pairs(pos, L, pl, pl->n * k / nch, pl->n * (k + 1) / nch, rc, ushift, fo,
                        &sums[2 * k], &sums[2 * k + 1]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 3 * n; q++)
        for (int k = 1; k < nch; k++) f[q] += fk[(size_t)(k - 1) * (size_t)n * 3 + q];
    double U = 0.0, W = 0.0;
    for (int k = 0; k < nch; k++) {
        U += sums[2 * k];
        W += sums[2 * k + 1];
    }
    *pe = U;
    *vir = W;
}

/* Forces through the cell lists (pairs within rc, no skin).  Returns 0 or -1. */
int orc_forces_cells(int64_t n, const double* pos, const double L[3], const int G[3], double rc,
                     double ushift, double* f, double* pe, double* vir)
{
    if (G[0] < 3 || G[1] < 3 || G[2] < 3) return -1;
    pairlist_t pl = {0, 0, 0};
    if (build_pairs_cells(n, pos, L, G, rc, &pl)) { free(pl.p); return -1; }
    double* fk = chunk_forces_alloc(n);
    forces_from_pairs(n, pos, L, &pl, rc, ushift, f, fk, pe, vir);
    free(fk);
    free(pl.p);
    return 0;
}

/* Direct O(N^2) minimum-image forces. */
void orc_forces_brute(int64_t n, const double* pos, const double L[3], double rc, double ushift,
                      double* f, double* pe, double* vir)
{
    double rc2 = rc * rc;
    double U = 0.0, W = 0.0;
    memset(f, 0, (size_t)n * 3 * sizeof(double));
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], L[0]);
            double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L[1]);
            double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2) {
                double fr, u;
                orc_pair(r2, ushift, &fr, &u);
                f[3 * i + 0] += fr * dx; f[3 * i + 1] += fr * dy; f[3 * i + 2] += fr * dz;
                f[3 * j + 0] -= fr * dx; f[3 * j + 1] -= fr * dy; f[3 * j + 2] -= fr * dz;
                U += u;
                W += fr * r2;
            }
        }
    *pe = U;
    *vir = W;
}

/* Force and potential energy share of selected atoms, each by a direct
 * O(N) minimum-image sum over all other atoms.  u_out[k] is the sum of u
 * over the pairs of atom idx[k] (so the total over all atoms is 2U).
 * Intended for spot checks of very large systems. */
void orc_forces_sampled(int64_t n, const double* pos, const double L[3], double rc, double ushift,
                        int64_t ns, const int64_t* idx, double* f_out, double* u_out)
{
    double rc2 = rc * rc;
    for (int64_t k = 0; k < ns; k++) {
        int64_t i = idx[k];
        double fx = 0, fy = 0, fz = 0, us = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = min_image(pos[3 * i + 0] - pos[3 * j + 0], L[0]);
            double dy = min_image(pos[3 * i + 1] - pos[3 * j + 1], L[1]);
            double dz = min_image(pos[3 * i + 2] - pos[3 * j + 2], L[2]);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rc2) {
                double fr, u;
                orc_pair(r2, ushift, &fr, &u);
                fx += fr * dx; fy += fr * dy; fz += fr * dz;
                us += u;
            }
        }
        f_out[3 * k + 0] = fx;
        f_out[3 * k + 1] = fy;
        f_out[3 * k + 2] = fz;
        u_out[k] = us;
    }
}

/* Atoms j != i within rcut of atom i by a direct O(N) minimum-image scan.
 * Writes up to cap indices (ascending) and returns the count. */
int64_t orc_neighbors_of(int64_t n, const double* pos, const double L[3], double rcut, int64_t i,
                         int64_t cap, int64_t* out)
{
    double rc2 = rcut * rcut;
    int64_t m = 0;
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        if (orc_pair_r2(pos, L, i, j) < rc2) {
            if (m < cap) out[m] = j;
            m++;
        }
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* The MD loop (Sec. 3.1, steps (a)-(f))                               */
/* ------------------------------------------------------------------ */

typedef struct {
    double L[3];
    double rc, skin, dt, ushift;
    int even_cells;
    int rescale_every;          /* step (f): 0 = off */
    int64_t rescale_until;      /* rescale while step <= rescale_until */
    double T_target;
} orc_params_t;

static double kinetic(int64_t n, const double* vel)
{
    double s = 0.0;
    for (int64_t i = 0; i < 3 * n; i++) s += vel[i] * vel[i];
    return 0.5 * s;
}

/* Runs nsteps velocity-Verlet steps from (pos, vel) with forces f(0)
 * computed first.  The neighbour list holds pairs within r_n = r_c + skin
 * and is rebuilt -- after wrapping positions into the region -- whenever the
 * largest displacement since the last rebuild reaches skin/2; with skin = 0
 * it is rebuilt every step (the cell-list-only variant).  Between rebuilds
 * positions are left unwrapped so stored shifts stay valid.
 *
 * Per-step records (index 0 = initial state, k = after step k), each
 * optional: ke, pe, vir (sum over pairs of r . f).  On return pos is wrapped
 * and f_out (optional) holds the final forces.  *nrebuild counts rebuilds
 * after the initial build; *npairs_sum accumulates the list length at each
 * build (initial included).  Returns 0, -1 (geometry) or -2 (memory). */
int orc_run(int64_t n, double* pos, double* vel, const orc_params_t* P, int64_t nsteps,
            double* ke, double* pe, double* vir, double* f_out, int64_t* nrebuild,
            int64_t* npairs_sum)
{
    int G[3];
    double rn = P->rc + P->skin;
    if (orc_cell_grid(P->L, rn, P->even_cells, G)) return -1;
    double* f = (double*)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double* xb = (double*)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double* fk = chunk_forces_alloc(n);
    if (!f || !xb || (n_chunks() > 1 && !fk)) { free(f); free(xb); free(fk); return -2; }
    pairlist_t pl = {0, 0, 0};
    double h = 0.5 * P->dt;
    double half_skin2 = 0.25 * P->skin * P->skin;
    int64_t nreb = 0, psum = 0;

    orc_wrap(n, pos, P->L);
    if (build_pairs_cells(n, pos, P->L, G, rn, &pl)) { free(f); free(xb); free(fk); free(pl.p); return -2; }
    psum += pl.n;
    memcpy(xb, pos, (size_t)n * 3 * sizeof(double));
    double U, W;
    forces_from_pairs(n, pos, P->L, &pl, P->rc, P->ushift, f, fk, &U, &W);
    if (ke) ke[0] = kinetic(n, vel);
    if (pe) pe[0] = U;
    if (vir) vir[0] = W;

    for (int64_t step = 1; step <= nsteps; step++) {
        /* (a) half kick, drift */
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < 3 * n; k++) {
            vel[k] = vel[k] + h * f[k];
            pos[k] = pos[k] + P->dt * vel[k];
        }
        /* (b) rebuild when the largest displacement reaches skin/2 */
        int far = 0;
#pragma omp parallel for schedule(static) reduction(| : far)
        for (int64_t i = 0; i < n; i++) {
            double dx = pos[3 * i + 0] - xb[3 * i + 0];
            double dy = pos[3 * i + 1] - xb[3 * i + 1];
            double dz = pos[3 * i + 2] - xb[3 * i + 2];
            if (dx * dx + dy * dy + dz * dz >= half_skin2) far = 1;
        }
        int rebuild = (P->skin == 0.0) || far;
        if (rebuild) {
            orc_wrap(n, pos, P->L);
            if (build_pairs_cells(n, pos, P->L, G, rn, &pl)) { free(f); free(xb); free(fk); free(pl.p); return -2; }
            psum += pl.n;
            memcpy(xb, pos, (size_t)n * 3 * sizeof(double));
            nreb++;
        }
        /* (c) forces */
        forces_from_pairs(n, pos, P->L, &pl, P->rc, P->ushift, f, fk, &U, &W);
        /* (d) half kick */
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < 3 * n; k++) vel[k] = vel[k] + h * f[k];
        /* (e) properties */
        if (ke) ke[step] = kinetic(n, vel);
        if (pe) pe[step] = U;
        if (vir) vir[step] = W;
        /* (f) equilibration: rescale to the target temperature */
        if (P->rescale_every > 0 && step <= P->rescale_until && step % P->rescale_every == 0) {
            double K = kinetic(n, vel);
            if (K > 0.0) {
                double s = sqrt(1.5 * (double)n * P->T_target / K);
                for (int64_t k = 0; k < 3 * n; k++) vel[k] *= s;
            }
        }
    }
    orc_wrap(n, pos, P->L);
    if (f_out) memcpy(f_out, f, (size_t)n * 3 * sizeof(double));
    if (nrebuild) *nrebuild = nreb;
    if (npairs_sum) *npairs_sum = psum;
    free(f); free(xb); free(fk); free(pl.p);
    return 0;
}
