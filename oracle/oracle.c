/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the docking hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * includes, links or calls it, and this file includes nothing of the CUDA
 * library: the two share no code, header, table or constant.
 *
 * What it computes (paper, Section II-A): a ligand is a set of atoms whose
 * pose is given by a genotype (translation, orientation, torsion angles of its
 * rotatable bonds); its energy is the particle-grid interaction read from
 * precomputed receptor grids plus the ligand's self-interactions (van der
 * Waals, hydrogen bonding, electrostatics, desolvation); a genetic algorithm
 * with crossover, fitness-based selection and a memetic local search on a
 * random sample of each generation (Lamarckian write-back) minimises it over
 * several independent runs of population 150; the answer is the best pose
 * over all runs.  The paper prints none of the functional forms or constants:
 * every form below is a reading (the AutoDock4 family's 12-6 / 12-10 pair
 * potentials, Mehler-Solmajer dielectric, Gaussian desolvation) and every
 * constant is defined by this project.  The local search is ADADELTA (Zeiler 2012),
 * which the paper reaches only through its citation of gradient-based local
 * search in AutoDock-GPU; the paper's own miniapp uses Solis-Wets, which
 * orc_solis_wets restates (Solis and Wets 1981, adaptive step with a bias
 * term) as the second local-search method.
 *
 * Precision: energies, forces, poses, gradients and ADADELTA in FP64.  The
 * genetic operators act on FP32 genes with explicitly rounded FP32 operations
 * (one IEEE single operation per step, no contraction), because their outputs
 * must be bit-identical to the GPU's given the same energies; compile with
 * -ffp-contract=off.
 *
 * Parity status: every function below is pinned by a CPU test except
 * orc_dock's final best-energy values, which are a stochastic search result:
 * their parity is "parity unpinned" beyond the brute-force bound and the
 * distribution comparison.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_ATOMS 256
#define ORC_MAX_TORS 32
#define ORC_NTYPES 7

/* ------------------------------------------------------------------------ */
/* Force-field readings (Section II-A names the terms only).                 */

typedef struct {
    double R;      /* A, pair radius contribution: R_ij = (R_i + R_j)/2 */
    double eps;    /* kcal/mol, eps_ij = sqrt(eps_i eps_j)               */
    double vol;    /* A^3, desolvation volume                            */
    double solpar; /* atomic solvation parameter                         */
    int hb;        /* 0 none, 1 donor, 2 acceptor                        */
    double Rhb;    /* A, 12-10 minimum for an acceptor paired with HD    */
    double ehb;    /* kcal/mol, 12-10 well depth for an acceptor         */
} orc_type_t;

/* C, A, N, NA, OA, SA, HD */
static const orc_type_t OT[ORC_NTYPES] = {
    {4.0, 0.15, 33.5, -0.0015, 0, 0.0, 0.0},
    {4.0, 0.15, 33.5, -0.0005, 0, 0.0, 0.0},
    {3.5, 0.16, 22.5, -0.0015, 0, 0.0, 0.0},
    {3.5, 0.16, 22.5, -0.0015, 2, 1.9, 5.0},
    {3.2, 0.20, 17.0, -0.0025, 2, 1.9, 5.0},
    {4.0, 0.20, 33.5, -0.0020, 2, 2.5, 1.0},
    {2.0, 0.02, 0.0, 0.0005, 1, 0.0, 0.0},
};

static const double W_VDW = 0.16, W_HB = 0.12, W_EL = 0.14, W_DS = 0.13;
static const double Q_SOLV = 0.011;      /* charge-dependent solvation factor */
static const double COULOMB = 332.06;    /* kcal A / (mol e^2)                */
/* Sigmoidal distance-dependent dielectric, Mehler & Solmajer (1991) form.   */
static const double DIEL_A = -8.5525, DIEL_EPS0 = 78.4, DIEL_LAMBDA = 0.003627, DIEL_K = 7.7839;
static const double DS_SIGMA = 3.6;      /* A, desolvation Gaussian width     */
static const double CUTOFF = 8.0;        /* A, intramolecular hard cutoff     */
static const double R_FLOOR = 0.5;       /* A, distances are floored here     */
static const double K_OUT = 10.0;        /* kcal/mol/A^2, out-of-box penalty  */
static const double MAP_CAP = 1.0e5;     /* cap on type-map values            */

/* ------------------------------------------------------------------------ */
/* Pair energy terms as functions of distance (Section II-A: van der Waals,  */
/* hydrogen bonding, electrostatics, desolvation).  Each returns E(r_eff)     */
/* and dE/dr, with r_eff = max(r, R_FLOOR); dE/dr = 0 below the floor.        */

static int is_hbond(int ta, int tb) {
    return (OT[ta].hb == 1 && OT[tb].hb == 2) || (OT[ta].hb == 2 && OT[tb].hb == 1);
}

/* 12-6 Lennard-Jones with minimum -eps_ij at R_ij, or 12-10 H-bond with
 * minimum -ehb at Rhb of the acceptor; weights included. */
double orc_vdw_hb(int ta, int tb, double r, double *dEdr) {
    double re = r < R_FLOOR ? R_FLOOR : r;
    double r2 = re * re, r6 = r2 * r2 * r2, r10 = r6 * r2 * r2, r12 = r6 * r6; /* re^n */
    double e, d;
    if (is_hbond(ta, tb)) {
        const orc_type_t *acc = OT[ta].hb == 2 ? &OT[ta] : &OT[tb];
        double R2 = acc->Rhb * acc->Rhb, R10 = R2 * R2 * R2 * R2 * R2;
        double c12 = 5.0 * acc->ehb * R10 * R2;
        double c10 = 6.0 * acc->ehb * R10;
        e = W_HB * (c12 / r12 - c10 / r10);
        d = W_HB * (-12.0 * c12 / (r12 * re) + 10.0 * c10 / (r10 * re));
    } else {
        double R = 0.5 * (OT[ta].R + OT[tb].R), R6 = R * R * R * R * R * R;
        double eps = sqrt(OT[ta].eps * OT[tb].eps);
        double c12 = eps * R6 * R6;
        double c6 = 2.0 * eps * R6;
        e = W_VDW * (c12 / r12 - c6 / r6);
        d = W_VDW * (-12.0 * c12 / (r12 * re) + 6.0 * c6 / (r6 * re));
    }
    if (dEdr) *dEdr = r < R_FLOOR ? 0.0 : d;
    return e;
}

double orc_dielectric(double r, double *deps) {
    double B = DIEL_EPS0 - DIEL_A;
    double ex = exp(-DIEL_LAMBDA * B * r);
    double den = 1.0 + DIEL_K * ex;
    if (deps) *deps = B * DIEL_K * DIEL_LAMBDA * B * ex / (den * den);
    return DIEL_A + B / den;
}

/* Screened Coulomb term w_el * 332.06 * qa qb / (eps(r) r). */
double orc_elec(double qa, double qb, double r, double *dEdr) {
    double re = r < R_FLOOR ? R_FLOOR : r;
    double de;
    double eps = orc_dielectric(re, &de);
    double c = W_EL * COULOMB * qa * qb;
    double e = c / (eps * re);
    if (dEdr) *dEdr = r < R_FLOOR ? 0.0 : -c * (eps + re * de) / ((eps * re) * (eps * re));
    return e;
}

static double solv(int t, double q) { return OT[t].solpar + Q_SOLV * fabs(q); }

/* Desolvation w_ds (S_a V_b + S_b V_a) exp(-r^2 / (2 sigma^2)). */
double orc_desolv(int ta, double qa, int tb, double qb, double r, double *dEdr) {
    double re = r < R_FLOOR ? R_FLOOR : r;
    double coef = W_DS * (solv(ta, qa) * OT[tb].vol + solv(tb, qb) * OT[ta].vol);
    double e = coef * exp(-re * re / (2.0 * DS_SIGMA * DS_SIGMA));
    if (dEdr) *dEdr = r < R_FLOOR ? 0.0 : -e * re / (DS_SIGMA * DS_SIGMA);
    return e;
}

/* Full intramolecular pair energy; zero at and beyond the 8 A cutoff. */
double orc_pair_energy(int ta, double qa, int tb, double qb, double r, double *dEdr) {
    if (r >= CUTOFF) {
        if (dEdr) *dEdr = 0.0;
        return 0.0;
    }
    double d1, d2, d3;
    double e = orc_vdw_hb(ta, tb, r, &d1) + orc_elec(qa, qb, r, &d2) + orc_desolv(ta, qa, tb, qb, r, &d3);
    if (dEdr) *dEdr = d1 + d2 + d3;
    return e;
}

/* ------------------------------------------------------------------------ */
/* Receptor grid maps: the "reaction field for the protein" of Section II-A.  */
/* Map t (ligand type t) at point p holds the interaction a neutral-charge-    */
/* part atom of type t would feel; the electrostatic map holds the potential   */
/* per unit ligand charge; the desolvation map the term per unit |charge|.    */
/* Atom energy = M_t(x) + q E(x) + |q| D(x).  No cutoff; type maps capped.    */

void orc_map_values_at(int nrec, const double *rxyz, const int *rtype, const double *rq,
                       int ntmaps, const int *map_types, double px, double py, double pz, double *out) {
    double *acc = out;
    for (int m = 0; m < ntmaps + 2; ++m) acc[m] = 0.0;
    for (int j = 0; j < nrec; ++j) {
        double dx = px - rxyz[3 * j], dy = py - rxyz[3 * j + 1], dz = pz - rxyz[3 * j + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double re = r < R_FLOOR ? R_FLOOR : r;
        int tj = rtype[j];
        double g = exp(-re * re / (2.0 * DS_SIGMA * DS_SIGMA));
        for (int m = 0; m < ntmaps; ++m) {
            int t = map_types[m];
            double e = orc_vdw_hb(t, tj, r, NULL);
            e += W_DS * (OT[t].solpar * OT[tj].vol + solv(tj, rq[j]) * OT[t].vol) * g;
            acc[m] += e;
        }
        acc[ntmaps] += orc_elec(1.0, rq[j], r, NULL);
        acc[ntmaps + 1] += W_DS * Q_SOLV * OT[tj].vol * g;
    }
    for (int m = 0; m < ntmaps; ++m)
        if (acc[m] > MAP_CAP) acc[m] = MAP_CAP;
}

typedef struct {
    int nrec;
    const double *rxyz;
    const int *rtype;
    const double *rq;
    int nx, ny, nz;
    double ox, oy, oz, h;
    int ntmaps;
    const int *map_types;
    double *out;
    int z0, z1;
} map_job_t;

static void *map_worker(void *arg) {
    map_job_t *J = (map_job_t *)arg;
    int nm = J->ntmaps + 2;
    double vals[ORC_NTYPES + 2];
    size_t plane = (size_t)J->nx * J->ny, vol = plane * J->nz;
    for (int z = J->z0; z < J->z1; ++z)
        for (int y = 0; y < J->ny; ++y)
            for (int x = 0; x < J->nx; ++x) {
                orc_map_values_at(J->nrec, J->rxyz, J->rtype, J->rq, J->ntmaps, J->map_types,
                                  J->ox + x * J->h, J->oy + y * J->h, J->oz + z * J->h, vals);
                for (int m = 0; m < nm; ++m) J->out[m * vol + z * plane + (size_t)y * J->nx + x] = vals[m];
            }
    return NULL;
}

/* All maps at every grid point; out is [ntmaps+2][nz][ny][nx], x fastest. */
int orc_build_maps(int nrec, const double *rxyz, const int *rtype, const double *rq, int nx, int ny, int nz,
                   double ox, double oy, double oz, double h, int ntmaps, const int *map_types, int nthreads,
                   double *out) {
    if (ntmaps < 1 || ntmaps > ORC_NTYPES || nx < 2 || ny < 2 || nz < 2 || h <= 0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nz) nthreads = nz;
    map_job_t jobs[256];
    pthread_t th[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; ++t) {
        map_job_t J = {nrec, rxyz, rtype, rq, nx, ny, nz, ox, oy, oz, h, ntmaps, map_types, out,
                       (int)((long)nz * t / nthreads), (int)((long)nz * (t + 1) / nthreads)};
        jobs[t] = J;
        pthread_create(&th[t], NULL, map_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid reads: trilinear interpolation (particle-grid interaction, II-A).     */

typedef struct {
    const float *maps; /* [nmaps][nz][ny][nx] FP32 values */
    int nx, ny, nz, nmaps;
    double ox, oy, oz, h;
    int map_of_type[8]; /* ligand type code -> map index, -1 if absent */
    int emap, dmap;
} orc_grid;

static double node(const orc_grid *g, int m, int x, int y, int z) {
    return (double)g->maps[(((size_t)m * g->nz + z) * g->ny + y) * g->nx + x];
}

/* Value of map m at (x,y,z) A and its gradient (A^-1 units).  Each grid
 * coordinate u = (x - origin)/h is clamped to [0, n-1]; along a clamped axis
 * the interpolation does not vary, so that gradient component is zero.  The
 * cell is i0 = min(floor(u), n-2), f = u - i0, so f = 1 on the upper face. */
double orc_interp(const orc_grid *g, int m, double x, double y, double z, double *grad) {
    double u[3] = {(x - g->ox) / g->h, (y - g->oy) / g->h, (z - g->oz) / g->h};
    int n[3] = {g->nx, g->ny, g->nz};
    int i0[3], clamped[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        clamped[a] = 0;
        if (u[a] < 0.0) { u[a] = 0.0; clamped[a] = 1; }
        if (u[a] > n[a] - 1) { u[a] = n[a] - 1; clamped[a] = 1; }
        int i = (int)floor(u[a]);
        if (i > n[a] - 2) i = n[a] - 2;
        i0[a] = i;
        f[a] = u[a] - i;
    }
    double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int c = 0; c < 8; ++c) {
        int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
        double wx = bx ? f[0] : 1.0 - f[0];
        double wy = by ? f[1] : 1.0 - f[1];
        double wz = bz ? f[2] : 1.0 - f[2];
        double val = node(g, m, i0[0] + bx, i0[1] + by, i0[2] + bz);
        v += wx * wy * wz * val;
        gx += (bx ? 1.0 : -1.0) * wy * wz * val;
        gy += wx * (by ? 1.0 : -1.0) * wz * val;
        gz += wx * wy * (bz ? 1.0 : -1.0) * val;
    }
    if (grad) {
        grad[0] = clamped[0] ? 0.0 : gx / g->h;
        grad[1] = clamped[1] ? 0.0 : gy / g->h;
        grad[2] = clamped[2] ? 0.0 : gz / g->h;
    }
    return v;
}

/* Quadratic penalty k_out d^2 per axis for the distance d (A) outside the
 * box spanned by the grid points. */
static double out_of_box(const orc_grid *g, const double *x, double *grad) {
    double lo[3] = {g->ox, g->oy, g->oz};
    int n[3] = {g->nx, g->ny, g->nz};
    double e = 0.0;
    for (int a = 0; a < 3; ++a) {
        double hi = lo[a] + (n[a] - 1) * g->h;
        double gr = 0.0;
        if (x[a] < lo[a]) {
            double d = lo[a] - x[a];
            e += K_OUT * d * d;
            gr = -2.0 * K_OUT * d;
        } else if (x[a] > hi) {
            double d = x[a] - hi;
            e += K_OUT * d * d;
            gr = 2.0 * K_OUT * d;
        }
        if (grad) grad[a] = gr;
    }
    return e;
}

/* Intermolecular energy of one ligand atom of type t, charge q at x. */
double orc_atom_grid_energy(const orc_grid *g, int t, double q, const double *x, double *grad) {
    double gm[3], ge[3], gd[3], gp[3];
    int m = g->map_of_type[t];
    if (m < 0) return NAN;
    double e = orc_interp(g, m, x[0], x[1], x[2], gm) + q * orc_interp(g, g->emap, x[0], x[1], x[2], ge) +
               fabs(q) * orc_interp(g, g->dmap, x[0], x[1], x[2], gd) + out_of_box(g, x, gp);
    if (grad)
        for (int a = 0; a < 3; ++a) grad[a] = gm[a] + q * ge[a] + fabs(q) * gd[a] + gp[a];
    return e;
}

/* ------------------------------------------------------------------------ */
/* Ligand model (Section II-A: atoms; rotatable bonds plus the rigid-body     */
/* motion are the degrees of freedom).                                         */

typedef struct {
    int n, nb, nt;
    double ref[ORC_MAX_ATOMS][3]; /* reference coordinates minus their centroid */
    int type[ORC_MAX_ATOMS];
    double q[ORC_MAX_ATOMS];
    int frag[ORC_MAX_ATOMS];      /* rigid fragment of each atom */
    int nfrag, root;
    int tors_a[ORC_MAX_TORS], tors_b[ORC_MAX_TORS]; /* a: root side, b: moving side */
    int tors_depth[ORC_MAX_TORS];
    unsigned char moves[ORC_MAX_TORS][ORC_MAX_ATOMS]; /* atom i turns with torsion k */
    int npairs;
    int *pi, *pj;
} orc_lig;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ECONN = -2, ORC_ERING = -3, ORC_ESIZE = -4, ORC_ETYPE = -5 };

static int reach(int n, int nb, const int *bonds, int skip, int start, unsigned char *seen, int only_rigid,
                 const int *rot) {
    int stack[ORC_MAX_ATOMS], sp = 0, cnt = 0;
    memset(seen, 0, (size_t)n);
    stack[sp++] = start;
    seen[start] = 1;
    while (sp) {
        int a = stack[--sp];
        ++cnt;
        for (int b = 0; b < nb; ++b) {
            if (b == skip || (only_rigid && rot[b])) continue;
            int u = bonds[2 * b], v = bonds[2 * b + 1], w = -1;
            if (u == a) w = v;
            else if (v == a) w = u;
            if (w >= 0 && !seen[w]) { seen[w] = 1; stack[sp++] = w; }
        }
    }
    return cnt;
}

int orc_ligand_create(int n, const double *xyz, const int *type, const double *q, int nb, const int *bonds,
                      const int *rot, orc_lig **out) {
    *out = NULL;
    if (n < 1 || n > ORC_MAX_ATOMS - 1) return ORC_ESIZE;
    for (int i = 0; i < n; ++i)
        if (type[i] < 0 || type[i] >= ORC_NTYPES) return ORC_ETYPE;
    for (int b = 0; b < nb; ++b) {
        int u = bonds[2 * b], v = bonds[2 * b + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return ORC_EINVAL;
    }
    orc_lig *L = (orc_lig *)calloc(1, sizeof(orc_lig));
    unsigned char seen[ORC_MAX_ATOMS];
    L->n = n;
    L->nb = nb;
    if (reach(n, nb, bonds, -1, 0, seen, 0, rot) != n) { free(L); return ORC_ECONN; }
    int nt = 0;
    for (int b = 0; b < nb; ++b) {
        if (!rot[b]) continue;
        if (nt == ORC_MAX_TORS) { free(L); return ORC_ESIZE; }
        /* A rotatable bond must be a bridge: removing it splits the graph. */
        if (reach(n, nb, bonds, b, bonds[2 * b], seen, 0, rot) == n) { free(L); return ORC_ERING; }
        L->tors_a[nt] = bonds[2 * b];
        L->tors_b[nt] = bonds[2 * b + 1];
        ++nt;
    }
    L->nt = nt;
    /* Reference conformation about its centroid. */
    double c[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) c[a] += xyz[3 * i + a];
    for (int a = 0; a < 3; ++a) c[a] /= n;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) L->ref[i][a] = xyz[3 * i + a] - c[a];
        L->type[i] = type[i];
        L->q[i] = q[i];
    }
    /* Rigid fragments: components over non-rotatable bonds. */
    for (int i = 0; i < n; ++i) L->frag[i] = -1;
    int nf = 0, fsize[ORC_MAX_ATOMS];
    for (int i = 0; i < n; ++i) {
        if (L->frag[i] >= 0) continue;
        fsize[nf] = reach(n, nb, bonds, -1, i, seen, 1, rot);
        for (int j = 0; j < n; ++j)
            if (seen[j]) L->frag[j] = nf;
        ++nf;
    }
    L->nfrag = nf;
    /* Root: the largest fragment; on a tie the one holding the lowest atom
     * index, which is the lower fragment number by construction. */
    int root = 0;
    for (int f = 1; f < nf; ++f)
        if (fsize[f] > fsize[root]) root = f;
    L->root = root;
    int root_atom = 0;
    while (L->frag[root_atom] != root) ++root_atom;
    /* Orientation of each torsion and the atoms it moves: removing bond k,
     * the side not holding the root fragment turns. */
    int tk = 0;
    for (int b = 0; b < nb; ++b) {
        if (!rot[b]) continue;
        reach(n, nb, bonds, b, root_atom, seen, 0, rot);
        int u = bonds[2 * b], v = bonds[2 * b + 1];
        if (seen[u]) { L->tors_a[tk] = u; L->tors_b[tk] = v; }
        else { L->tors_a[tk] = v; L->tors_b[tk] = u; }
        for (int i = 0; i < n; ++i) L->moves[tk][i] = !seen[i];
        ++tk;
    }
    /* Depth of torsion k: number of rotatable bonds between the root and the
     * moving side, i.e. the torsions whose moving set contains b_k. */
    for (int k = 0; k < nt; ++k) {
        int d = 0;
        for (int j = 0; j < nt; ++j)
            if (L->moves[j][L->tors_b[k]]) ++d;
        L->tors_depth[k] = d; /* >= 1: k moves its own b */
    }
    /* Bond-graph distances by breadth-first search. */
    int *dist = (int *)malloc(sizeof(int) * n * n);
    for (int s = 0; s < n; ++s) {
        int *ds = dist + s * n, queue[ORC_MAX_ATOMS], qh = 0, qt = 0;
        for (int i = 0; i < n; ++i) ds[i] = -1;
        ds[s] = 0;
        queue[qt++] = s;
        while (qh < qt) {
            int a = queue[qh++];
            for (int b = 0; b < nb; ++b) {
                int u = bonds[2 * b], v = bonds[2 * b + 1], w = -1;
                if (u == a) w = v;
                else if (v == a) w = u;
                if (w >= 0 && ds[w] < 0) { ds[w] = ds[a] + 1; queue[qt++] = w; }
            }
        }
    }
    /* Pair list: atoms in different rigid fragments, separated by >= 4 bonds
     * (1-2, 1-3 and 1-4 neighbours excluded). */
    L->pi = (int *)malloc(sizeof(int) * (n * (n - 1) / 2 + 1));
    L->pj = (int *)malloc(sizeof(int) * (n * (n - 1) / 2 + 1));
    L->npairs = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (L->frag[i] != L->frag[j] && dist[i * n + j] >= 4) {
                L->pi[L->npairs] = i;
                L->pj[L->npairs] = j;
                ++L->npairs;
            }
    free(dist);
    *out = L;
    return ORC_OK;
}

void orc_ligand_free(orc_lig *L) {
    if (!L) return;
    free(L->pi);
    free(L->pj);
    free(L);
}

int orc_ligand_info(const orc_lig *L, int *nt, int *npairs, int *nfrag) {
    *nt = L->nt;
    *npairs = L->npairs;
    *nfrag = L->nfrag;
    return 0;
}

int orc_ligand_pairs(const orc_lig *L, int *ij) {
    for (int p = 0; p < L->npairs; ++p) {
        ij[2 * p] = L->pi[p];
        ij[2 * p + 1] = L->pj[p];
    }
    return L->npairs;
}

int orc_ligand_torsion(const orc_lig *L, int k, int *a, int *b, int *depth, unsigned char *moves) {
    if (k < 0 || k >= L->nt) return -1;
    *a = L->tors_a[k];
    *b = L->tors_b[k];
    *depth = L->tors_depth[k];
    memcpy(moves, L->moves[k], (size_t)L->n);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Genotype -> pose (Section IV-B: atom rotations applied in a fixed order).  */

/* Rotation of v about unit axis u by angle th (right-hand rule, Rodrigues). */
static void rodrigues(const double *u, double th, const double *v, double *out) {
    double c = cos(th), s = sin(th);
    double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double d = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    for (int a = 0; a < 3; ++a) out[a] = v[a] * c + cr[a] * s + u[a] * d * (1.0 - c);
}

static void apply_torsion(const orc_lig *L, int k, double th, double (*p)[3]) {
    const double *A = p[L->tors_a[k]], *B = p[L->tors_b[k]];
    double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) u[a] /= len;
    double b[3] = {B[0], B[1], B[2]};
    for (int i = 0; i < L->n; ++i) {
        if (!L->moves[k][i]) continue;
        double v[3] = {p[i][0] - b[0], p[i][1] - b[1], p[i][2] - b[2]}, w[3];
        rodrigues(u, th, v, w);
        for (int a = 0; a < 3; ++a) p[i][a] = b[a] + w[a];
    }
}

/* Internal conformation: the centred reference with torsion deltas applied.
 * order 0: deepest torsion first (ties: lower index first), each about its
 * axis in the coordinates current at that point -- the reading used by the
 * scorer.  order 1: root-most first with moving axes; both give the same
 * conformation, which a test checks. */
int orc_pose_local(const orc_lig *L, const double *tau, int order, double *out) {
    double (*p)[3] = (double (*)[3])out;
    for (int i = 0; i < L->n; ++i)
        for (int a = 0; a < 3; ++a) p[i][a] = L->ref[i][a];
    int maxd = 0;
    for (int k = 0; k < L->nt; ++k)
        if (L->tors_depth[k] > maxd) maxd = L->tors_depth[k];
    for (int s = 0; s < maxd; ++s) {
        int d = order == 0 ? maxd - s : s + 1;
        for (int k = 0; k < L->nt; ++k)
            if (L->tors_depth[k] == d) apply_torsion(L, k, tau[k], p);
    }
    return 0;
}

/* Unit-quaternion rotation matrix for q = (w, x, y, z). */
static void quat_matrix(const double *q, double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Genotype (t[3], q[4] unnormalised, tau[T]) -> atom coordinates [n][3]:
 * x_i = t + R(q/|q|) p_i(tau).  Returns |q|. */
double orc_pose(const orc_lig *L, const double *geno, double *xyz) {
    double p[ORC_MAX_ATOMS][3], R[3][3];
    orc_pose_local(L, geno + 7, 0, &p[0][0]);
    double nq = sqrt(geno[3] * geno[3] + geno[4] * geno[4] + geno[5] * geno[5] + geno[6] * geno[6]);
    double qh[4] = {1, 0, 0, 0};
    if (nq >= 1e-12)
        for (int a = 0; a < 4; ++a) qh[a] = geno[3 + a] / nq;
    quat_matrix(qh, R);
    for (int i = 0; i < L->n; ++i)
        for (int a = 0; a < 3; ++a)
            xyz[3 * i + a] = geno[a] + R[a][0] * p[i][0] + R[a][1] * p[i][1] + R[a][2] * p[i][2];
    return nq;
}

/* ------------------------------------------------------------------------ */
/* Energy of coordinates and of genotypes, with the analytic gradient.        */

/* Intramolecular energy of arbitrary coordinates (pair list, cutoff); adds
 * dE/dx into f when f is given. */
double orc_intra_xyz(const orc_lig *L, const double *xyz, double *f) {
    double e = 0.0;
    for (int p = 0; p < L->npairs; ++p) {
        int i = L->pi[p], j = L->pj[p];
        double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1], xyz[3 * i + 2] - xyz[3 * j + 2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dEdr;
        e += orc_pair_energy(L->type[i], L->q[i], L->type[j], L->q[j], r, &dEdr);
        if (f && dEdr != 0.0)
            for (int a = 0; a < 3; ++a) {
                f[3 * i + a] += dEdr * d[a] / r;
                f[3 * j + a] -= dEdr * d[a] / r;
            }
    }
    return e;
}

double orc_inter_xyz(const orc_lig *L, const orc_grid *g, const double *xyz, double *f) {
    double e = 0.0, gr[3];
    for (int i = 0; i < L->n; ++i) {
        e += orc_atom_grid_energy(g, L->type[i], L->q[i], xyz + 3 * i, gr);
        if (f)
            for (int a = 0; a < 3; ++a) f[3 * i + a] += gr[a];
    }
    return e;
}

/* E(genotype) and, when grad is given, dE/dgenotype:
 *   dE/dt      = sum_i f_i                                  (f_i = dE/dx_i)
 *   dE/dq      = 2 ((0, G) (x) qhat) / |q|,  G = sum_i (x_i - t) x f_i
 *   dE/dtau_k  = sum_{i moved by k} (u_k x (x_i - x_{b_k})) . f_i,
 *                u_k = unit(x_{b_k} - x_{a_k})
 * terms (optional): {intermolecular incl. penalty, intramolecular}. */
double orc_score(const orc_lig *L, const orc_grid *g, const double *geno, double *grad, double *xyz_out,
                 double *terms) {
    double x[ORC_MAX_ATOMS * 3], f[ORC_MAX_ATOMS * 3];
    double nq = orc_pose(L, geno, x);
    memset(f, 0, sizeof(double) * 3 * L->n);
    double ei = orc_inter_xyz(L, g, x, f);
    double ea = orc_intra_xyz(L, x, f);
    if (terms) { terms[0] = ei; terms[1] = ea; }
    if (xyz_out) memcpy(xyz_out, x, sizeof(double) * 3 * L->n);
    if (grad) {
        double F[3] = {0, 0, 0}, G[3] = {0, 0, 0};
        for (int i = 0; i < L->n; ++i) {
            double *fi = f + 3 * i;
            double d[3] = {x[3 * i] - geno[0], x[3 * i + 1] - geno[1], x[3 * i + 2] - geno[2]};
            for (int a = 0; a < 3; ++a) F[a] += fi[a];
            G[0] += d[1] * fi[2] - d[2] * fi[1];
            G[1] += d[2] * fi[0] - d[0] * fi[2];
            G[2] += d[0] * fi[1] - d[1] * fi[0];
        }
        for (int a = 0; a < 3; ++a) grad[a] = F[a];
        if (nq >= 1e-12) {
            double w = geno[3] / nq, qx = geno[4] / nq, qy = geno[5] / nq, qz = geno[6] / nq;
            /* (0, G) (x) (w, qx, qy, qz), Hamilton product */
            double pw = -G[0] * qx - G[1] * qy - G[2] * qz;
            double px = G[0] * w + G[1] * qz - G[2] * qy;
            double py = -G[0] * qz + G[1] * w + G[2] * qx;
            double pz = G[0] * qy - G[1] * qx + G[2] * w;
            grad[3] = 2.0 * pw / nq;
            grad[4] = 2.0 * px / nq;
            grad[5] = 2.0 * py / nq;
            grad[6] = 2.0 * pz / nq;
        } else {
            grad[3] = grad[4] = grad[5] = grad[6] = 0.0;
        }
        for (int k = 0; k < L->nt; ++k) {
            const double *A = x + 3 * L->tors_a[k], *B = x + 3 * L->tors_b[k];
            double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            double len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            for (int a = 0; a < 3; ++a) u[a] /= len;
            double s = 0.0;
            for (int i = 0; i < L->n; ++i) {
                if (!L->moves[k][i]) continue;
                double v[3] = {x[3 * i] - B[0], x[3 * i + 1] - B[1], x[3 * i + 2] - B[2]};
                double c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
                s += c[0] * f[3 * i] + c[1] * f[3 * i + 1] + c[2] * f[3 * i + 2];
            }
            grad[7 + k] = s;
        }
    }
    return ei + ea;
}

/* Distances of the pose from the places where the FP32 and FP64 answers may
 * legitimately differ: out[0] = smallest distance (grid units) of any atom
 * coordinate from a cell face, out[1] = smallest |r - 8 A| over pairs,
 * out[2] = smallest |r - r_floor| over pairs. */
void orc_pose_margins(const orc_lig *L, const orc_grid *g, const double *geno, double *out) {
    double x[ORC_MAX_ATOMS * 3];
    orc_pose(L, geno, x);
    double o[3] = {g->ox, g->oy, g->oz};
    double m0 = 1e300, m1 = 1e300, m2 = 1e300;
    for (int i = 0; i < L->n; ++i)
        for (int a = 0; a < 3; ++a) {
            double u = (x[3 * i + a] - o[a]) / g->h;
            double d = fabs(u - floor(u + 0.5));
            if (d < m0) m0 = d;
        }
    for (int p = 0; p < L->npairs; ++p) {
        int i = L->pi[p], j = L->pj[p];
        double d0 = x[3 * i] - x[3 * j], d1 = x[3 * i + 1] - x[3 * j + 1], d2 = x[3 * i + 2] - x[3 * j + 2];
        double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        if (fabs(r - CUTOFF) < m1) m1 = fabs(r - CUTOFF);
        if (fabs(r - R_FLOOR) < m2) m2 = fabs(r - R_FLOOR);
    }
    out[0] = m0;
    out[1] = m1;
    out[2] = m2;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its        */
/* published definition: ten rounds of two 32x32->64 multiplies with a Weyl   */
/* key schedule.                                                              */

void orc_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
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

/* Stream layout of the search: counter = (purpose << 16 | draw, entity,
 * generation, run), key = (seed low word, seed high word). */
enum { P_INIT = 1, P_SELECT = 2, P_CROSS = 3, P_MUTATE = 4, P_LSPICK = 5, P_SW = 6 };

static void draw4(uint64_t seed, uint32_t run, uint32_t gen, uint32_t entity, uint32_t purpose, uint32_t draw,
                  uint32_t *w) {
    uint32_t c[4] = {(purpose << 16) | draw, entity, gen, run};
    uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(c, k, w);
}

/* Uniform float in [0,1): the top 24 bits times 2^-24 (exact in FP32). */
static float unif(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }
/* Uniform index in [0, n): floor of the 24-bit fraction times n, in integers. */
static uint32_t uidx(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)(w >> 8) * n) >> 24); }

/* ------------------------------------------------------------------------ */
/* Genetic operators (Section II-A: crossover, fitness-based selection; the   */
/* rates and operator forms are this project's readings).  FP32 genes, every  */
/* arithmetic step one rounded IEEE single operation in a fixed order.        */

/* Solis-Wets constants (this project's readings): initial and lowest step
 * scale, expansion and contraction factors, the runs of consecutive
 * successes / failures that trigger them, and the deviation half-width per
 * gene block at scale 1 (translation in A, quaternion component, torsion in
 * radians). */
typedef struct {
    float rho0, rho_lo, expand, contract;
    int n_succ, n_fail;
    float step_t, step_q, step_tau;
} orc_sw_t;

typedef struct {
    int pop_size;
    int nruns;
    long long max_evals;
    int ls_count;   /* individuals given a local search per generation */
    int ls_iters;   /* iterations per local search (ADADELTA or Solis-Wets) */
    double rho, eps;
    float p_tour, p_cross, p_mut, trans_mut;
    int ls_method;  /* 0 = ADADELTA, 1 = Solis-Wets */
    orc_sw_t sw;
} orc_params;

static const float PI_F = 3.14159265358979323846f;
static const float TWO_PI_F = 6.28318530717958647692f;

static float wrap_f(float x) {
    if (x >= PI_F) x = x - TWO_PI_F;
    else if (x < -PI_F) x = x + TWO_PI_F;
    return x;
}

/* Search box in FP32: lo = origin, len = (n-1) h, both rounded once. */
static void box_f(const orc_grid *g, float *lo, float *len) {
    lo[0] = (float)g->ox; lo[1] = (float)g->oy; lo[2] = (float)g->oz;
    len[0] = (float)((g->nx - 1) * g->h);
    len[1] = (float)((g->ny - 1) * g->h);
    len[2] = (float)((g->nz - 1) * g->h);
}

/* Initial individual: translation uniform in the box, orientation uniform on
 * the unit 3-sphere by Marsaglia's (1972) two-disc method, torsions uniform
 * in [-pi, pi). */
void orc_init_individual(int nt, const orc_grid *g, uint64_t seed, uint32_t run, uint32_t slot, float *gene) {
    float lo[3], len[3];
    uint32_t w[4];
    box_f(g, lo, len);
    draw4(seed, run, 0, slot, P_INIT, 0, w);
    for (int a = 0; a < 3; ++a) gene[a] = lo[a] + unif(w[a]) * len[a];
    gene[3] = 1.0f; gene[4] = gene[5] = gene[6] = 0.0f;
    for (uint32_t att = 0; att < 32; ++att) {
        draw4(seed, run, 0, slot, P_INIT, 1 + att, w);
        float x1 = 2.0f * unif(w[0]) - 1.0f, x2 = 2.0f * unif(w[1]) - 1.0f;
        float x3 = 2.0f * unif(w[2]) - 1.0f, x4 = 2.0f * unif(w[3]) - 1.0f;
        float s1 = x1 * x1 + x2 * x2, s2 = x3 * x3 + x4 * x4;
        if (s1 < 1.0f && s2 < 1.0f && s2 > 0.0f) {
            float fct = sqrtf((1.0f - s1) / s2);
            gene[3] = x1; gene[4] = x2; gene[5] = x3 * fct; gene[6] = x4 * fct;
            break;
        }
    }
    for (int k = 0; k < nt; ++k) {
        if ((k & 3) == 0) draw4(seed, run, 0, slot, P_INIT, 64 + (uint32_t)(k >> 2), w);
        gene[7 + k] = unif(w[k & 3]) * TWO_PI_F - PI_F;
    }
}

/* Binary tournament: two uniform picks, the fitter (lower energy; on a tie the
 * lower index) wins with probability p_tour. */
static int tournament(const double *E, int pop, float p_tour, const uint32_t *w) {
    int i1 = (int)uidx(w[0], (uint32_t)pop), i2 = (int)uidx(w[1], (uint32_t)pop);
    int better, worse;
    if (E[i1] < E[i2] || (E[i1] == E[i2] && i1 <= i2)) { better = i1; worse = i2; }
    else { better = i2; worse = i1; }
    return unif(w[2]) < p_tour ? better : worse;
}

/* Next generation of one run.  Slot 0 takes the best individual (elitism;
 * lowest index on a tie).  Each slot s >= 1: parents by two tournaments,
 * two-point crossover over gene blocks (tx, ty, tz, quaternion, each torsion)
 * with probability p_cross, then per-block mutation with probability p_mut.
 * info (optional) gets per slot: parent1, parent2, cut lo, cut hi, mutated
 * block mask (bit b).  Returns the elite index. */
int orc_ga_children(int nt, int pop, const float *pop_old, const double *E_old, uint64_t seed, uint32_t run,
                    uint32_t gen, const orc_params *P, float *pop_new, long long *info) {
    int G = 7 + nt, nblk = 4 + nt;
    int elite = 0;
    for (int i = 1; i < pop; ++i)
        if (E_old[i] < E_old[elite]) elite = i;
    memcpy(pop_new, pop_old + (size_t)elite * G, sizeof(float) * G);
    if (info) { info[0] = elite; info[1] = elite; info[2] = 0; info[3] = 0; info[4] = 0; }
    for (int s = 1; s < pop; ++s) {
        uint32_t w[4];
        draw4(seed, run, gen, (uint32_t)s, P_SELECT, 0, w);
        int p1 = tournament(E_old, pop, P->p_tour, w);
        draw4(seed, run, gen, (uint32_t)s, P_SELECT, 1, w);
        int p2 = tournament(E_old, pop, P->p_tour, w);
        draw4(seed, run, gen, (uint32_t)s, P_CROSS, 0, w);
        int lo = 0, hi = 0;
        if (unif(w[0]) < P->p_cross) {
            int c1 = (int)uidx(w[1], (uint32_t)nblk), c2 = (int)uidx(w[2], (uint32_t)nblk);
            lo = c1 < c2 ? c1 : c2;
            hi = c1 < c2 ? c2 : c1;
        }
        float *ch = pop_new + (size_t)s * G;
        const float *A = pop_old + (size_t)p1 * G, *B = pop_old + (size_t)p2 * G;
        /* block b -> genes: b<3: gene b; b==3: genes 3..6; b>=4: gene b+3 */
        for (int b = 0; b < nblk; ++b) {
            const float *src = (b >= lo && b < hi) ? B : A;
            if (b < 3) ch[b] = src[b];
            else if (b == 3) for (int a = 3; a < 7; ++a) ch[a] = src[a];
            else ch[b + 3] = src[b + 3];
        }
        long long mask = 0;
        for (int b = 0; b < nblk; ++b) {
            if ((b & 3) == 0) draw4(seed, run, gen, (uint32_t)s, P_MUTATE, (uint32_t)(b >> 2), w);
            if (unif(w[b & 3]) < P->p_mut) mask |= 1LL << b;
        }
        for (int b = 0; b < nblk; ++b) {
            if (!(mask >> b & 1)) continue;
            uint32_t v[4];
            draw4(seed, run, gen, (uint32_t)s, P_MUTATE, 16 + (uint32_t)b, v);
            if (b < 3) {
                float delta = unif(v[0]) * (2.0f * P->trans_mut) - P->trans_mut;
                ch[b] = ch[b] + delta;
            } else if (b == 3) {
                /* q <- normalise((1, v) (x) q), v uniform in [-1,1)^3 */
                float vx = 2.0f * unif(v[0]) - 1.0f, vy = 2.0f * unif(v[1]) - 1.0f, vz = 2.0f * unif(v[2]) - 1.0f;
                float qw = ch[3], qx = ch[4], qy = ch[5], qz = ch[6];
                float nw = ((qw - vx * qx) - vy * qy) - vz * qz;
                float nx = ((qx + vx * qw) + vy * qz) - vz * qy;
                float ny = ((qy - vx * qz) + vy * qw) + vz * qx;
                float nz = ((qz + vx * qy) - vy * qx) + vz * qw;
                float nrm = sqrtf(((nw * nw + nx * nx) + ny * ny) + nz * nz);
                ch[3] = nw / nrm; ch[4] = nx / nrm; ch[5] = ny / nrm; ch[6] = nz / nrm;
            } else {
                float delta = unif(v[0]) * TWO_PI_F - PI_F;
                ch[b + 3] = wrap_f(ch[b + 3] + delta);
            }
        }
        if (info) {
            long long *r = info + 5 * s;
            r[0] = p1; r[1] = p2; r[2] = lo; r[3] = hi; r[4] = mask;
        }
    }
    return elite;
}

/* The sample given a local search: the first ls_count entries of a partial
 * Fisher-Yates shuffle of 0..pop-1. */
void orc_ls_picks(int pop, int n_ls, uint64_t seed, uint32_t run, uint32_t gen, int *picks) {
    int *a = (int *)malloc(sizeof(int) * (size_t)(pop > 0 ? pop : 1));
    for (int i = 0; i < pop; ++i) a[i] = i;
    for (int k = 0; k < n_ls; ++k) {
        uint32_t w[4];
        draw4(seed, run, gen, (uint32_t)k, P_LSPICK, 0, w);
        int j = k + (int)uidx(w[0], (uint32_t)(pop - k));
        int t = a[k]; a[k] = a[j]; a[j] = t;
        picks[k] = a[k];
    }
    free(a);
}

/* Normalise the quaternion genes in FP32 (same op order as the mutation). */
static void normalise_q(float *ge) {
    float n = sqrtf(((ge[3] * ge[3] + ge[4] * ge[4]) + ge[5] * ge[5]) + ge[6] * ge[6]);
    if (n > 0.0f) { ge[3] = ge[3] / n; ge[4] = ge[4] / n; ge[5] = ge[5] / n; ge[6] = ge[6] / n; }
}

/* ------------------------------------------------------------------------ */
/* ADADELTA (Zeiler 2012) on the genotype; the local search of the memetic    */
/* step.  State starts at zero for every search; one iteration = one energy   */
/* and gradient evaluation at the current point, then one update; the best    */
/* point seen is kept (Lamarckian write-back of the best, not the last).       */

static double wrap_d(double x) {
    const double tp = 2.0 * M_PI;
    return x - tp * floor((x + M_PI) / tp);
}

void orc_adadelta_step(int G, int nt, double rho, double eps, double *x, const double *g, double *Eg2, double *Edx2) {
    for (int j = 0; j < G; ++j) {
        Eg2[j] = rho * Eg2[j] + (1.0 - rho) * g[j] * g[j];
        double dx = -sqrt(Edx2[j] + eps) / sqrt(Eg2[j] + eps) * g[j];
        Edx2[j] = rho * Edx2[j] + (1.0 - rho) * dx * dx;
        x[j] += dx;
    }
    for (int k = 0; k < nt; ++k) x[7 + k] = wrap_d(x[7 + k]);
}

double orc_local_search(const orc_lig *L, const orc_grid *g, const float *x0, int iters, double rho, double eps,
                        float *x_out, double *trace) {
    int G = 7 + L->nt;
    double x[7 + ORC_MAX_TORS], gr[7 + ORC_MAX_TORS], Eg2[7 + ORC_MAX_TORS], Edx2[7 + ORC_MAX_TORS];
    double best[7 + ORC_MAX_TORS], Ebest = INFINITY;
    for (int j = 0; j < G; ++j) { x[j] = x0[j]; Eg2[j] = 0.0; Edx2[j] = 0.0; best[j] = x0[j]; }
    for (int it = 0; it < iters; ++it) {
        double E = orc_score(L, g, x, gr, NULL, NULL);
        if (trace) trace[it] = E;
        if (E < Ebest) { Ebest = E; memcpy(best, x, sizeof(double) * G); }
        orc_adadelta_step(G, L->nt, rho, eps, x, gr, Eg2, Edx2);
    }
    double n = sqrt(best[3] * best[3] + best[4] * best[4] + best[5] * best[5] + best[6] * best[6]);
    for (int j = 0; j < G; ++j) x_out[j] = (float)((j >= 3 && j < 7 && n > 0) ? best[j] / n : best[j]);
    return Ebest;
}

/* ------------------------------------------------------------------------ */
/* Solis-Wets local search (Solis and Wets 1981, the adaptive random search   */
/* with a bias term), the memetic step of the paper's miniapp (Section II-A). */
/* State: the current point x (always the best seen), its energy, a bias b    */
/* (start 0), a step scale rho (start rho0) and the runs of consecutive       */
/* successes and failures.  One iteration draws a deviation                   */
/*     xi_j = b_j + rho * step(block of j) * u_j,   u_j uniform in [-1, 1)     */
/* and tries x + xi; if that is not lower it tries x - xi.  A success moves   */
/* x there and sets b <- 0.2 b + 0.4 xi (forward) or b <- b - 0.4 xi          */
/* (backward); a failure halves b.  n_succ successes in a row multiply rho    */
/* by expand, n_fail failures in a row by contract (either resets both runs). */
/* The search ends after iters iterations or once rho < rho_lo.  Genes, xi,   */
/* b and rho are FP32, each step one rounded single operation, so that given  */
/* the same accept decisions the GPU reproduces every point bit for bit;      */
/* energies are FP64.  u_j is word j mod 4 of the Philox block              */
/* (P_SW << 16 | 10 it + j / 4, entity, gen, run).                              */

static double score_f(const orc_lig *L, const orc_grid *g, const float *ge);

/* torsion wrap to [-pi, pi) for any finite x, FP32 single operations */
static float wrap_any_f(float x) {
    float k = floorf((x + PI_F) / TWO_PI_F);
    return x - TWO_PI_F * k;
}

static float sw_step_of(const orc_sw_t *S, int j) {
    return j < 3 ? S->step_t : (j < 7 ? S->step_q : S->step_tau);
}

/* E0: energy of x0 (NaN: evaluated here, one evaluation).  trace (optional,
 * [iters][4]): energy of x + xi, of x - xi (NaN if not tried), rho used and
 * the outcome (+1 forward success, -1 backward success, 0 failure); rows
 * after the last iteration are left untouched.  Returns the final energy;
 * x_out = final point, quaternion normalised; *evals = energies computed. */
double orc_solis_wets(const orc_lig *L, const orc_grid *g, const float *x0, double E0, int iters,
                      const orc_sw_t *S, uint64_t seed, uint32_t run, uint32_t gen, uint32_t entity,
                      float *x_out, long long *evals, double *trace, int *iters_done) {
    const int G = 7 + L->nt;
    float x[7 + ORC_MAX_TORS], b[7 + ORC_MAX_TORS], xi[7 + ORC_MAX_TORS], y[7 + ORC_MAX_TORS];
    long long n = 0;
    for (int j = 0; j < G; ++j) { x[j] = x0[j]; b[j] = 0.0f; }
    double E = E0;
    if (isnan(E)) { E = score_f(L, g, x); ++n; }
    float rho = S->rho0;
    int ns = 0, nf = 0, it = 0;
    for (; it < iters && rho >= S->rho_lo; ++it) {
        uint32_t w[4];
        for (int j = 0; j < G; ++j) {
            if ((j & 3) == 0) draw4(seed, run, gen, entity, P_SW, (uint32_t)(10 * it + j / 4), w);
            float u = 2.0f * unif(w[j & 3]) - 1.0f;
            xi[j] = b[j] + (rho * sw_step_of(S, j)) * u;
        }
        for (int j = 0; j < G; ++j) y[j] = x[j] + xi[j];
        for (int k = 7; k < G; ++k) y[k] = wrap_any_f(y[k]);
        double Ef = score_f(L, g, y), Eb = NAN;
        ++n;
        int outcome = 0;
        if (Ef < E) {
            memcpy(x, y, sizeof(float) * G);
            E = Ef;
            for (int j = 0; j < G; ++j) b[j] = 0.2f * b[j] + 0.4f * xi[j];
            outcome = 1;
        } else {
            for (int j = 0; j < G; ++j) y[j] = x[j] - xi[j];
            for (int k = 7; k < G; ++k) y[k] = wrap_any_f(y[k]);
            Eb = score_f(L, g, y);
            ++n;
            if (Eb < E) {
                memcpy(x, y, sizeof(float) * G);
                E = Eb;
                for (int j = 0; j < G; ++j) b[j] = b[j] - 0.4f * xi[j];
                outcome = -1;
            } else {
                for (int j = 0; j < G; ++j) b[j] = 0.5f * b[j];
            }
        }
        if (trace) {
            trace[4 * it] = Ef;
            trace[4 * it + 1] = Eb;
            trace[4 * it + 2] = rho;
            trace[4 * it + 3] = outcome;
        }
        if (outcome) { ++ns; nf = 0; } else { ++nf; ns = 0; }
        if (ns >= S->n_succ) { rho = rho * S->expand; ns = 0; }
        else if (nf >= S->n_fail) { rho = rho * S->contract; nf = 0; }
    }
    memcpy(x_out, x, sizeof(float) * G);
    normalise_q(x_out);
    if (evals) *evals = n;
    if (iters_done) *iters_done = it;
    return E;
}

/* ------------------------------------------------------------------------ */
/* The Lamarckian GA over independent runs (Section II-A).  Per generation:   */
/* children (elitism, tournaments, crossover, mutation) and their energies;   */
/* a local search (ADADELTA or Solis-Wets) on ls_count individuals drawn     */
/* without replacement, written back; evaluation count += (pop-1) + the       */
/* energies the local searches computed (the per-run sum of Listing 1:        */
/* ls_count*ls_iters for ADADELTA).  Stops at the first generation boundary   */
/* with evals >= max_evals.                                                   */

typedef struct {
    const orc_lig *L;
    const orc_grid *g;
    const orc_params *P;
    uint64_t seed;
    int run;
    float *best_geno;
    double *best_E;
    long long *evals;
} run_job_t;

static double score_f(const orc_lig *L, const orc_grid *g, const float *ge) {
    double x[7 + ORC_MAX_TORS];
    for (int j = 0; j < 7 + L->nt; ++j) x[j] = ge[j];
    return orc_score(L, g, x, NULL, NULL, NULL);
}

static void run_lga(run_job_t *J) {
    const orc_lig *L = J->L;
    const orc_params *P = J->P;
    int G = 7 + L->nt, pop = P->pop_size;
    float *A = (float *)malloc(sizeof(float) * pop * G), *B = (float *)malloc(sizeof(float) * pop * G);
    double *EA = (double *)malloc(sizeof(double) * pop), *EB = (double *)malloc(sizeof(double) * pop);
    int *picks = (int *)malloc(sizeof(int) * (P->ls_count > 0 ? P->ls_count : 1));
    for (int s = 0; s < pop; ++s) {
        orc_init_individual(L->nt, J->g, J->seed, (uint32_t)J->run, (uint32_t)s, A + (size_t)s * G);
        EA[s] = score_f(L, J->g, A + (size_t)s * G);
    }
    long long evals = pop;
    uint32_t gen = 0;
    while (evals < P->max_evals) {
        ++gen;
        int elite = orc_ga_children(L->nt, pop, A, EA, J->seed, (uint32_t)J->run, gen, P, B, NULL);
        EB[0] = EA[elite];
        for (int s = 1; s < pop; ++s) EB[s] = score_f(L, J->g, B + (size_t)s * G);
        orc_ls_picks(pop, P->ls_count, J->seed, (uint32_t)J->run, gen, picks);
        long long ls_evals = 0;
        for (int k = 0; k < P->ls_count; ++k) {
            float *ind = B + (size_t)picks[k] * G;
            if (P->ls_method == 1) {
                long long n = 0;
                EB[picks[k]] = orc_solis_wets(L, J->g, ind, EB[picks[k]], P->ls_iters, &P->sw, J->seed,
                                              (uint32_t)J->run, gen, (uint32_t)k, ind, &n, NULL, NULL);
                ls_evals += n;
            } else {
                EB[picks[k]] = orc_local_search(L, J->g, ind, P->ls_iters, P->rho, P->eps, ind, NULL);
                ls_evals += P->ls_iters;
            }
        }
        evals += (pop - 1) + ls_evals;
        float *t = A; A = B; B = t;
        double *te = EA; EA = EB; EB = te;
    }
    int best = 0;
    for (int s = 1; s < pop; ++s)
        if (EA[s] < EA[best]) best = s;
    memcpy(J->best_geno, A + (size_t)best * G, sizeof(float) * G);
    normalise_q(J->best_geno);
    *J->best_E = score_f(L, J->g, J->best_geno);
    *J->evals = evals;
    free(A); free(B); free(EA); free(EB); free(picks);
}

typedef struct {
    run_job_t *jobs;
    int njobs;
    int next;
    pthread_mutex_t mu;
} run_pool_t;

static void *run_worker(void *arg) {
    run_pool_t *R = (run_pool_t *)arg;
    for (;;) {
        pthread_mutex_lock(&R->mu);
        int k = R->next++;
        pthread_mutex_unlock(&R->mu);
        if (k >= R->njobs) return NULL;
        run_lga(&R->jobs[k]);
    }
}

/* Runs P->nruns independent searches, one per thread up to nthreads.  The
 * result of each run does not depend on nthreads. */
int orc_dock(const orc_lig *L, const orc_grid *g, const orc_params *P, uint64_t seed, int nthreads,
             float *best_geno, double *best_E, long long *evals) {
    if (P->pop_size < 2 || P->ls_count < 0 || P->ls_count > P->pop_size || P->nruns < 1) return ORC_EINVAL;
    if (P->ls_method == 1 && P->ls_iters > 6553) return ORC_EINVAL;  /* 10 it + 9 must fit 16 bits */
    int G = 7 + L->nt;
    run_job_t *jobs = (run_job_t *)malloc(sizeof(run_job_t) * P->nruns);
    for (int r = 0; r < P->nruns; ++r) {
        run_job_t J = {L, g, P, seed, r, best_geno + (size_t)r * G, best_E + r, evals + r};
        jobs[r] = J;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > P->nruns) nthreads = P->nruns;
    run_pool_t R;
    R.jobs = jobs;
    R.njobs = P->nruns;
    R.next = 0;
    pthread_mutex_init(&R.mu, NULL);
    pthread_t th[512];
    if (nthreads > 512) nthreads = 512;
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, run_worker, &R);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&R.mu);
    free(jobs);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Batch helpers for the tests: B genotypes (FP32 genes, as stored by a       */
/* population), energies and gradients in FP64, spread over threads.         */

typedef struct {
    const orc_lig *L;
    const orc_grid *g;
    const float *geno;
    double *E, *grad;
    int b0, b1;
} batch_job_t;

static void *batch_worker(void *arg) {
    batch_job_t *J = (batch_job_t *)arg;
    int G = 7 + J->L->nt;
    double x[7 + ORC_MAX_TORS];
    for (int b = J->b0; b < J->b1; ++b) {
        for (int j = 0; j < G; ++j) x[j] = J->geno[(size_t)b * G + j];
        J->E[b] = orc_score(J->L, J->g, x, J->grad ? J->grad + (size_t)b * G : NULL, NULL, NULL);
    }
    return NULL;
}

int orc_score_batch(const orc_lig *L, const orc_grid *g, const float *geno, int B, double *E, double *grad,
                    int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > B) nthreads = B > 0 ? B : 1;
    batch_job_t jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        batch_job_t J = {L, g, geno, E, grad, (int)((long)B * t / nthreads), (int)((long)B * (t + 1) / nthreads)};
        jobs[t] = J;
        pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

void orc_init_population(int nt, const orc_grid *g, uint64_t seed, uint32_t run, int pop, float *out) {
    for (int s = 0; s < pop; ++s) orc_init_individual(nt, g, seed, run, (uint32_t)s, out + (size_t)s * (7 + nt));
}

/* dE/dx_i of every atom (input order, [n][3]) at the pose of a genotype;
 * returns E.  Used to bound how much an FP32 rounding of the atom positions
 * can move the energy: |dE| <= sum_i |f_i|_1 * |dx|_max. */
double orc_atom_forces(const orc_lig *L, const orc_grid *g, const double *geno, double *f_out) {
    double x[ORC_MAX_ATOMS * 3];
    orc_pose(L, geno, x);
    memset(f_out, 0, sizeof(double) * 3 * L->n);
    return orc_inter_xyz(L, g, x, f_out) + orc_intra_xyz(L, x, f_out);
}
