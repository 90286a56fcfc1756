/*
 * pv_oracle.c -- plain, slow, FP64 CPU oracle for the PocketVina docking hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, call or execute this file;
 * only the test suite, the smoke check and the CPU-baseline leg of the benchmark do. It shares
 * no code, header, table or constant with the CUDA implementation: every constant below is
 * typed here from its source.
 *
 * What it computes, in the paper's order (arxiv 2506.20043, Methods "Accelerated Docking with
 * QuickVina 2-GPU 2.1", Eq. 1-13, Supplementary Algorithm 2; "PocketVina", Algorithm 3):
 *   - grid cache G_t over the receptor, one map per ligand atom type (Kernel 1),
 *   - POT conformations (Eq. 1), random start, one-entity mutation (Eq. 2),
 *   - SF = e_inter + e_intra (Eq. 3), e_inter by trilinear interpolation of G_t,
 *   - analytic gradient of SF over the pose tangent space,
 *   - RILC-BFGS: two-loop L-BFGS (Eq. 6, 9-11), Lewis-Overton line search (Eq. 7-8),
 *     termination (Eq. 12),
 *   - Metropolis acceptance (Eq. 13, read as exp((e_cur - e_new)/T), T = 1.2),
 *     refinement of a new best,
 *   - per-thread best output, sort + RMSD filter + top-k (Algorithm 2).
 *
 * The paper does not print the pairwise terms; they are the published AutoDock Vina terms
 * (Trott & Olson 2010, cited by the paper for the Vina family): gauss1, gauss2, repulsion,
 * hydrophobic, hydrogen bond on the surface distance d = r - R_i - R_j, 8 A cutoff.
 *
 * Readings where the paper is silent (each is one constant or one rule here):
 *   grid nodes origin + i*spacing, i = 0..ceil(size/spacing); atoms outside the grid are
 *   interpolated at the clamped point plus K_OUT * (distance outside); intra pairs are those
 *   in different rigid fragments more than three bonds apart; m = 5 pairs of L-BFGS memory;
 *   eps = 1e-3 for both Eq. 11 and Eq. 12; at most 10 line-search trials; iteration budget
 *   floor((25 + N_atoms) / 3); mutation amplitude 2 A (translation) and 2/R_gyr rad
 *   (orientation), torsion redrawn uniformly; RMSD filter 1 A.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011), written here from that definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ---------------------------------------------------------------- constants (Vina 2010) --- */
enum { XS_C_H = 0, XS_C_P, XS_N_P, XS_N_D, XS_N_A, XS_N_DA, XS_O_P, XS_O_D, XS_O_A, XS_O_DA,
       XS_S_P, XS_NTYPES };

static const double W_GAUSS1 = -0.0356;
static const double W_GAUSS2 = -0.00516;
static const double W_REPULSION = 0.840;
static const double W_HYDROPHOBIC = -0.0351;
static const double W_HBOND = -0.587;
static const double W_ROT = 0.0585;
static const double CUTOFF = 8.0;
static const double K_OUT = 10.0;        /* kcal/mol/A, outside-grid penalty slope (reading) */
static const double RECEPTOR_POLAR_C_DIST = 1.75; /* C is polar if an N/O lies this close   */

static double xs_radius(int t) {
    switch (t) {
        case XS_C_H: case XS_C_P: return 1.9;
        case XS_N_P: case XS_N_D: case XS_N_A: case XS_N_DA: return 1.8;
        case XS_O_P: case XS_O_D: case XS_O_A: case XS_O_DA: return 1.7;
        default: return 2.0; /* S_P */
    }
}
static int xs_hydrophobic(int t) { return t == XS_C_H; }
static int xs_donor(int t) { return t == XS_N_D || t == XS_N_DA || t == XS_O_D || t == XS_O_DA; }
static int xs_acceptor(int t) { return t == XS_N_A || t == XS_N_DA || t == XS_O_A || t == XS_O_DA; }

/* ------------------------------------------------------------------------ Philox4x32-10 --- */
/* One round: two 32x32->64 multiplies, xor with the other counter words and the key. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

/* Draw stream of one chain at one step: word i is word (i mod 4) of
 * philox(ctr = {chain, unit, step, i / 4}, key = {seed lo, seed hi}). */
typedef struct { uint32_t chain, unit, step; uint64_t seed; } or_stream;

static uint32_t stream_word(const or_stream* s, int i) {
    uint32_t ctr[4] = {s->chain, s->unit, s->step, (uint32_t)(i / 4)};
    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[i % 4];
}
/* Uniform in [0, 1) from the top 24 bits: exact in binary32 and binary64 alike. */
static double stream_uniform(const or_stream* s, int i) {
    return (double)(stream_word(s, i) >> 8) * (1.0 / 16777216.0);
}
double or_u01(uint32_t word) { return (double)(word >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------- small vector math --- */
static void v_sub(const double a[3], const double b[3], double o[3]) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double v_dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void v_cross(const double a[3], const double b[3], double o[3]) {
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static double v_norm(const double a[3]) { return sqrt(v_dot(a, a)); }

/* Rotation matrix of the unit quaternion (w, x, y, z), Hamilton convention. */
static void quat_to_mat(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
static void mat_vec(const double R[9], const double v[3], double o[3]) {
    double t0 = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    double t1 = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    double t2 = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static void quat_mul(const double a[4], const double b[4], double o[4]) {
    double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}
/* q <- normalize(exp(omega / 2) (x) q): rotate by the rotation vector omega in the world frame. */
static void quat_rotate_by(double q[4], const double omega[3]) {
    double th = v_norm(omega), e[4];
    if (th < 1e-14) {
        e[0] = 1.0; e[1] = 0.5 * omega[0]; e[2] = 0.5 * omega[1]; e[3] = 0.5 * omega[2];
    } else {
        double s = sin(0.5 * th) / th;
        e[0] = cos(0.5 * th); e[1] = s * omega[0]; e[2] = s * omega[1]; e[3] = s * omega[2];
    }
    double o[4];
    quat_mul(e, q, o);
    double n = sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + o[3] * o[3]);
    for (int k = 0; k < 4; ++k) q[k] = o[k] / n;
}
/* Rodrigues: rotate v about the unit axis a by angle t. */
static void rodrigues(const double a[3], double t, const double v[3], double o[3]) {
    double c = cos(t), s = sin(t), axv[3];
    v_cross(a, v, axv);
    double adv = v_dot(a, v);
    for (int k = 0; k < 3; ++k) o[k] = v[k] * c + axv[k] * s + a[k] * adv * (1 - c);
}

/* ------------------------------------------------------------------------- XS typing --- */
/* Elements 0 C, 1 N, 2 O, 3 S. Ligand carbon is polar iff bonded to N or O (Vina). */
void or_xs_type_ligand(int n, const uint8_t* elem, const uint8_t* don, const uint8_t* acc,
                       int nb, const int32_t* bonds, int32_t* out) {
    for (int i = 0; i < n; ++i) {
        int e = elem[i], t;
        if (e == 0) {
            int polar = 0;
            for (int b = 0; b < nb; ++b) {
                int o = -1;
                if (bonds[2 * b] == i) o = bonds[2 * b + 1];
                if (bonds[2 * b + 1] == i) o = bonds[2 * b];
                if (o >= 0 && (elem[o] == 1 || elem[o] == 2)) polar = 1;
            }
            t = polar ? XS_C_P : XS_C_H;
        } else if (e == 1) {
            t = XS_N_P + (don[i] ? 1 : 0) + (acc[i] ? 2 : 0);
        } else if (e == 2) {
            t = XS_O_P + (don[i] ? 1 : 0) + (acc[i] ? 2 : 0);
        } else {
            t = XS_S_P;
        }
        out[i] = t;
    }
}

/* Receptor carbons carry no bonds here: polar iff an N or O lies within 1.75 A. */
void or_xs_type_receptor(int n, const double* xyz, const uint8_t* elem, const uint8_t* don,
                         const uint8_t* acc, int32_t* out) {
    for (int i = 0; i < n; ++i) {
        int e = elem[i], t;
        if (e == 0) {
            int polar = 0;
            for (int j = 0; j < n; ++j) {
                if (j == i || !(elem[j] == 1 || elem[j] == 2)) continue;
                double d[3];
                v_sub(xyz + 3 * i, xyz + 3 * j, d);
                if (v_norm(d) < RECEPTOR_POLAR_C_DIST) polar = 1;
            }
            t = polar ? XS_C_P : XS_C_H;
        } else if (e == 1) {
            t = XS_N_P + (don[i] ? 1 : 0) + (acc[i] ? 2 : 0);
        } else if (e == 2) {
            t = XS_O_P + (don[i] ? 1 : 0) + (acc[i] ? 2 : 0);
        } else {
            t = XS_S_P;
        }
        out[i] = t;
    }
}

/* ----------------------------------------------------------------- pairwise Vina terms --- */
/* Unweighted terms at surface distance d: gauss1, gauss2, repulsion, hydrophobic, hbond. */
void or_terms(double d, double out[5]) {
    out[0] = exp(-(d / 0.5) * (d / 0.5));
    out[1] = exp(-((d - 3.0) / 2.0) * ((d - 3.0) / 2.0));
    out[2] = d < 0 ? d * d : 0.0;
    out[3] = d < 0.5 ? 1.0 : (d < 1.5 ? 1.5 - d : 0.0);
    out[4] = d < -0.7 ? 1.0 : (d < 0 ? -d / 0.7 : 0.0);
}
/* Their derivatives with respect to d (one-sided choice at the kinks: value of the piece
 * that holds at d itself). */
static void terms_deriv(double d, double out[5]) {
    out[0] = -2.0 * d / 0.25 * exp(-(d / 0.5) * (d / 0.5));
    out[1] = -2.0 * (d - 3.0) / 4.0 * exp(-((d - 3.0) / 2.0) * ((d - 3.0) / 2.0));
    out[2] = d < 0 ? 2.0 * d : 0.0;
    out[3] = d < 0.5 ? 0.0 : (d < 1.5 ? -1.0 : 0.0);
    out[4] = d < -0.7 ? 0.0 : (d < 0 ? -1.0 / 0.7 : 0.0);
}

/* Weighted energy of one atom pair of XS types ti, tj at distance r, and dE/dr. */
double or_pair_energy(int ti, int tj, double r, double* dedr) {
    if (dedr) *dedr = 0.0;
    if (r >= CUTOFF) return 0.0;
    double d = r - xs_radius(ti) - xs_radius(tj);
    double f[5], df[5];
    or_terms(d, f);
    terms_deriv(d, df);
    double hyd = (xs_hydrophobic(ti) && xs_hydrophobic(tj)) ? 1.0 : 0.0;
    double hb = ((xs_donor(ti) && xs_acceptor(tj)) || (xs_acceptor(ti) && xs_donor(tj))) ? 1.0 : 0.0;
    double e = W_GAUSS1 * f[0] + W_GAUSS2 * f[1] + W_REPULSION * f[2] + W_HYDROPHOBIC * hyd * f[3]
             + W_HBOND * hb * f[4];
    if (dedr)
        *dedr = W_GAUSS1 * df[0] + W_GAUSS2 * df[1] + W_REPULSION * df[2]
              + W_HYDROPHOBIC * hyd * df[3] + W_HBOND * hb * df[4];
    return e;
}

/* ----------------------------------------------------------------------- grid cache --- */
/* Kernel 1 of the paper: G_t(node) = sum over receptor atoms j of E(t, type_j, |node - x_j|).
 * Brute force over every receptor atom; no cells, no capping. */
int or_grid_dims(double size, double spacing) {
    return (int)ceil(size / spacing - 1e-9) + 1;
}

double or_grid_node_value(int n_rec, const double* rxyz, const int32_t* rtype, const double origin[3],
                          double spacing, int t, int ix, int iy, int iz) {
    double p[3] = {origin[0] + ix * spacing, origin[1] + iy * spacing, origin[2] + iz * spacing};
    double acc = 0.0;
    for (int j = 0; j < n_rec; ++j) {
        double d[3];
        v_sub(p, rxyz + 3 * j, d);
        acc += or_pair_energy(t, rtype[j], v_norm(d), NULL);
    }
    return acc;
}

/* Full maps, layout [map][z][y][x] (x fastest); map k is ligand XS type types[k]. */
void or_grid_build(int n_rec, const double* rxyz, const int32_t* rtype, const double origin[3],
                   double spacing, const int32_t dims[3], int n_maps, const int32_t* types,
                   double* maps, int n_threads) {
    long nx = dims[0], ny = dims[1], nz = dims[2];
    long nn = nx * ny * nz;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (long node = 0; node < nn; ++node) {
        int ix = (int)(node % nx), iy = (int)((node / nx) % ny), iz = (int)(node / (nx * ny));
        for (int m = 0; m < n_maps; ++m)
            maps[m * nn + node] = or_grid_node_value(n_rec, rxyz, rtype, origin, spacing, types[m],
                                                     ix, iy, iz);
    }
    (void)n_threads;
}

/* The same maps, filled only at the listed flat node indices (the rest untouched): lets a test
 * check a full-size workload on the nodes that sampled poses actually touch. */
void or_grid_fill_nodes(int n_rec, const double* rxyz, const int32_t* rtype, const double origin[3],
                        double spacing, const int32_t dims[3], int n_maps, const int32_t* types,
                        long n_nodes, const int64_t* nodes, double* maps, int n_threads) {
    long nx = dims[0], ny = dims[1], nz = dims[2];
    long nn = nx * ny * nz;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long k = 0; k < n_nodes; ++k) {
        long node = nodes[k];
        int ix = (int)(node % nx), iy = (int)((node / nx) % ny), iz = (int)(node / (nx * ny));
        for (int m = 0; m < n_maps; ++m)
            maps[m * nn + node] = or_grid_node_value(n_rec, rxyz, rtype, origin, spacing, types[m],
                                                     ix, iy, iz);
    }
    (void)nz;
    (void)n_threads;
}

typedef struct {
    double origin[3];
    double spacing;
    int32_t dims[3];
    int32_t map_of_type[XS_NTYPES]; /* -1 where the type has no map */
    const double* maps;             /* [n_maps][z][y][x] */
} or_grid;

/* Trilinear interpolation of the map of type t at point p (Eq. 3: e_inter from the grid cache)
 * and its gradient. Outside the grid: value at the clamped point plus K_OUT * distance. */
double or_grid_eval(const or_grid* G, int t, const double p[3], double dEdx[3]) {
    int m = G->map_of_type[t];
    long nx = G->dims[0], ny = G->dims[1], nz = G->dims[2];
    const double* V = G->maps + (long)m * nx * ny * nz;
    double gc[3], f[3], out[3];
    int i[3], clamped[3];
    for (int k = 0; k < 3; ++k) {
        double g = (p[k] - G->origin[k]) / G->spacing;
        double hi = (double)(G->dims[k] - 1);
        clamped[k] = (g < 0.0) || (g > hi);
        gc[k] = g < 0.0 ? 0.0 : (g > hi ? hi : g);
        i[k] = (int)floor(gc[k]);
        if (i[k] > G->dims[k] - 2) i[k] = G->dims[k] - 2;
        f[k] = gc[k] - i[k];
        out[k] = clamped[k] ? p[k] - (G->origin[k] + gc[k] * G->spacing) : 0.0;
    }
    double val = 0.0, dg[3] = {0, 0, 0};
    for (int c = 0; c < 8; ++c) {
        int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
        double v = V[((long)(i[2] + e) * ny + (i[1] + b)) * nx + (i[0] + a)];
        double wx = a ? f[0] : 1 - f[0], wy = b ? f[1] : 1 - f[1], wz = e ? f[2] : 1 - f[2];
        val += wx * wy * wz * v;
        dg[0] += (a ? 1.0 : -1.0) * wy * wz * v;
        dg[1] += wx * (b ? 1.0 : -1.0) * wz * v;
        dg[2] += wx * wy * (e ? 1.0 : -1.0) * v;
    }
    for (int k = 0; k < 3; ++k) dEdx[k] = clamped[k] ? 0.0 : dg[k] / G->spacing;
    double dist = v_norm(out);
    if (dist > 0.0) {
        val += K_OUT * dist;
        for (int k = 0; k < 3; ++k) dEdx[k] += K_OUT * out[k] / dist;
    }
    return val;
}

/* --------------------------------------------------------------------- ligand tree --- */
typedef struct {
    int n, nb, n_rot, n_frag, root, origin, n_pairs;
    double* ref;        /* [n][3] input conformer (psi = 0) */
    int32_t* xs;        /* [n] */
    int32_t* frag_of;   /* [n] rigid fragment id */
    int32_t* tor_p;     /* [n_rot] root-side atom of torsion k (k-th rotatable bond, input order) */
    int32_t* tor_c;     /* [n_rot] far-side atom */
    uint8_t* moves;     /* [n_rot][n] atom i is on the far side of torsion k */
    int32_t* order;     /* [n_rot] torsions sorted root-outward */
    int32_t* pairs;     /* [n_pairs][2] intra pairs */
    double rgyr;
} or_ligand;

static int uf_find(int* par, int x) {
    while (par[x] != x) x = par[x] = par[par[x]];
    return x;
}

void or_ligand_free(or_ligand* L) {
    if (!L) return;
    free(L->ref); free(L->xs); free(L->frag_of); free(L->tor_p); free(L->tor_c);
    free(L->moves); free(L->order); free(L->pairs); free(L);
}

/* Builds the torsion tree. Returns NULL if a rotatable bond is not a bridge (it would close a
 * ring of fragments). Torsion k is the k-th rotatable bond in input order. */
or_ligand* or_ligand_new(int n, const double* xyz, const uint8_t* elem, const uint8_t* don,
                         const uint8_t* acc, int nb, const int32_t* bonds, const uint8_t* rot) {
    or_ligand* L = (or_ligand*)calloc(1, sizeof(or_ligand));
    L->n = n; L->nb = nb;
    L->ref = (double*)malloc(sizeof(double) * 3 * n);
    memcpy(L->ref, xyz, sizeof(double) * 3 * n);
    L->xs = (int32_t*)malloc(sizeof(int32_t) * n);
    or_xs_type_ligand(n, elem, don, acc, nb, bonds, L->xs);

    /* rigid fragments: components over non-rotatable bonds */
    int* par = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) par[i] = i;
    for (int b = 0; b < nb; ++b)
        if (!rot[b]) par[uf_find(par, bonds[2 * b])] = uf_find(par, bonds[2 * b + 1]);
    L->frag_of = (int32_t*)malloc(sizeof(int32_t) * n);
    int* rep_to_frag = (int*)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) rep_to_frag[i] = -1;
    int nf = 0;
    for (int i = 0; i < n; ++i) {
        int r = uf_find(par, i);
        if (rep_to_frag[r] < 0) rep_to_frag[r] = nf++;
        L->frag_of[i] = rep_to_frag[r];
    }
    L->n_frag = nf;
    /* root: the fragment with most atoms; ties to the fragment holding the lowest atom index
     * (fragments are numbered by their lowest atom, so the lowest id wins). */
    int* fsize = (int*)calloc(nf, sizeof(int));
    for (int i = 0; i < n; ++i) fsize[L->frag_of[i]]++;
    L->root = 0;
    for (int f = 1; f < nf; ++f)
        if (fsize[f] > fsize[L->root]) L->root = f;
    L->origin = -1;
    for (int i = 0; i < n && L->origin < 0; ++i)
        if (L->frag_of[i] == L->root) L->origin = i;

    /* torsions in input order; far side = atoms not reachable from the root fragment when
     * the bond is cut */
    int nr = 0;
    for (int b = 0; b < nb; ++b) nr += rot[b] ? 1 : 0;
    L->n_rot = nr;
    L->tor_p = (int32_t*)malloc(sizeof(int32_t) * (nr ? nr : 1));
    L->tor_c = (int32_t*)malloc(sizeof(int32_t) * (nr ? nr : 1));
    L->moves = (uint8_t*)calloc((size_t)(nr ? nr : 1) * n, 1);
    L->order = (int32_t*)malloc(sizeof(int32_t) * (nr ? nr : 1));
    int* seen = (int*)malloc(sizeof(int) * n);
    int* stack = (int*)malloc(sizeof(int) * n);
    int ok = 1, k = 0;
    for (int b = 0; b < nb && ok; ++b) {
        if (!rot[b]) continue;
        /* reachability from the origin without crossing bond b */
        for (int i = 0; i < n; ++i) seen[i] = 0;
        int sp = 0;
        stack[sp++] = L->origin; seen[L->origin] = 1;
        while (sp) {
            int a = stack[--sp];
            for (int e = 0; e < nb; ++e) {
                if (e == b) continue;
                int o = -1;
                if (bonds[2 * e] == a) o = bonds[2 * e + 1];
                if (bonds[2 * e + 1] == a) o = bonds[2 * e];
                if (o >= 0 && !seen[o]) { seen[o] = 1; stack[sp++] = o; }
            }
        }
        int a0 = bonds[2 * b], a1 = bonds[2 * b + 1];
        if (seen[a0] == seen[a1]) ok = 0; /* not a bridge */
        L->tor_p[k] = seen[a0] ? a0 : a1;
        L->tor_c[k] = seen[a0] ? a1 : a0;
        for (int i = 0; i < n; ++i) L->moves[(size_t)k * n + i] = seen[i] ? 0 : 1;
        ++k;
    }
    /* root-outward order: a torsion's depth is the number of torsions that move its far atom */
    if (ok) {
        int* depth = (int*)malloc(sizeof(int) * (nr ? nr : 1));
        for (int a = 0; a < nr; ++a) {
            depth[a] = 0;
            for (int j = 0; j < nr; ++j)
                if (j != a && L->moves[(size_t)j * n + L->tor_c[a]]) depth[a]++;
            L->order[a] = a;
        }
        for (int a = 1; a < nr; ++a) { /* insertion sort by (depth, index) */
            int v = L->order[a], j = a - 1;
            while (j >= 0 && depth[L->order[j]] > depth[v]) { L->order[j + 1] = L->order[j]; --j; }
            L->order[j + 1] = v;
        }
        free(depth);
    }
    /* intra pairs: different rigid fragments and more than three bonds apart */
    int* dist = (int*)malloc(sizeof(int) * n);
    int* queue = (int*)malloc(sizeof(int) * n);
    L->pairs = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(n * (n - 1) / 2 + 1));
    L->n_pairs = 0;
    for (int i = 0; i < n && ok; ++i) {
        for (int j = 0; j < n; ++j) dist[j] = -1;
        int qh = 0, qt = 0;
        queue[qt++] = i; dist[i] = 0;
        while (qh < qt) {
            int a = queue[qh++];
            for (int e = 0; e < nb; ++e) {
                int o = -1;
                if (bonds[2 * e] == a) o = bonds[2 * e + 1];
                if (bonds[2 * e + 1] == a) o = bonds[2 * e];
                if (o >= 0 && dist[o] < 0) { dist[o] = dist[a] + 1; queue[qt++] = o; }
            }
        }
        for (int j = i + 1; j < n; ++j) {
            if (L->frag_of[i] == L->frag_of[j]) continue;
            if (dist[j] >= 0 && dist[j] <= 3) continue;
            L->pairs[2 * L->n_pairs] = i;
            L->pairs[2 * L->n_pairs + 1] = j;
            L->n_pairs++;
        }
    }
    /* gyration radius of the input conformer about the origin atom */
    double acc2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double d[3];
        v_sub(L->ref + 3 * i, L->ref + 3 * L->origin, d);
        acc2 += v_dot(d, d);
    }
    L->rgyr = sqrt(acc2 / n);
    free(par); free(rep_to_frag); free(fsize); free(seen); free(stack); free(dist); free(queue);
    if (!ok) { or_ligand_free(L); return NULL; }
    return L;
}

/* info: n, n_rot, n_frag, root, origin, n_pairs */
void or_ligand_info(const or_ligand* L, int32_t out[6], double* rgyr) {
    out[0] = L->n; out[1] = L->n_rot; out[2] = L->n_frag; out[3] = L->root; out[4] = L->origin;
    out[5] = L->n_pairs;
    if (rgyr) *rgyr = L->rgyr;
}
void or_ligand_arrays(const or_ligand* L, int32_t* xs, int32_t* frag_of, int32_t* pairs,
                      int32_t* tor_p, int32_t* tor_c) {
    if (xs) memcpy(xs, L->xs, sizeof(int32_t) * L->n);
    if (frag_of) memcpy(frag_of, L->frag_of, sizeof(int32_t) * L->n);
    if (pairs) memcpy(pairs, L->pairs, sizeof(int32_t) * 2 * L->n_pairs);
    if (tor_p) memcpy(tor_p, L->tor_p, sizeof(int32_t) * L->n_rot);
    if (tor_c) memcpy(tor_c, L->tor_c, sizeof(int32_t) * L->n_rot);
}

/* ------------------------------------------------------------ forward kinematics (Eq. 1) --- */
/* POT = (x, y, z, qw, qx, qy, qz, psi_1..psi_Nrot). Torsions are applied root-outward, each
 * rotating its far side about its current bond axis (root side -> far side), right-handed; then
 * the rigid motion puts the origin atom at (x, y, z) with orientation q. */
void or_fk(const or_ligand* L, const double* pot, double* xyz) {
    int n = L->n;
    double* X = (double*)malloc(sizeof(double) * 3 * n);
    memcpy(X, L->ref, sizeof(double) * 3 * n);
    for (int a = 0; a < L->n_rot; ++a) {
        int k = L->order[a];
        double axis[3];
        v_sub(X + 3 * L->tor_c[k], X + 3 * L->tor_p[k], axis);
        double len = v_norm(axis);
        for (int c = 0; c < 3; ++c) axis[c] /= len;
        const double* piv = X + 3 * L->tor_c[k];
        double pv[3] = {piv[0], piv[1], piv[2]};
        for (int i = 0; i < n; ++i) {
            if (!L->moves[(size_t)k * n + i]) continue;
            double v[3], o[3];
            v_sub(X + 3 * i, pv, v);
            rodrigues(axis, pot[7 + k], v, o);
            for (int c = 0; c < 3; ++c) X[3 * i + c] = pv[c] + o[c];
        }
    }
    double R[9];
    quat_to_mat(pot + 3, R);
    const double* xo = X + 3 * L->origin;
    double o0[3] = {xo[0], xo[1], xo[2]};
    for (int i = 0; i < n; ++i) {
        double v[3], o[3];
        v_sub(X + 3 * i, o0, v);
        mat_vec(R, v, o);
        for (int c = 0; c < 3; ++c) xyz[3 * i + c] = pot[c] + o[c];
    }
    free(X);
}

/* ------------------------------------------------------- scoring function (Eq. 3) + grad --- */
/* SF = e_inter + e_intra. grad (optional, 6 + N_rot): d SF / d(translation), d SF / d(rotation
 * vector applied in the world frame about the origin atom), d SF / d psi_k. parts (optional):
 * e_inter, e_intra. */
double or_score(const or_ligand* L, const or_grid* G, const double* pot, double* grad, double* parts) {
    int n = L->n;
    double* x = (double*)malloc(sizeof(double) * 3 * n);
    double* dE = (double*)calloc(3 * (size_t)n, sizeof(double));
    or_fk(L, pot, x);
    double e_inter = 0.0, e_intra = 0.0;
    for (int i = 0; i < n; ++i) {
        double g[3];
        e_inter += or_grid_eval(G, L->xs[i], x + 3 * i, g);
        for (int c = 0; c < 3; ++c) dE[3 * i + c] += g[c];
    }
    for (int p = 0; p < L->n_pairs; ++p) {
        int i = L->pairs[2 * p], j = L->pairs[2 * p + 1];
        double d[3], dedr;
        v_sub(x + 3 * i, x + 3 * j, d);
        double r = v_norm(d);
        e_intra += or_pair_energy(L->xs[i], L->xs[j], r, &dedr);
        if (r > 0.0)
            for (int c = 0; c < 3; ++c) {
                dE[3 * i + c] += dedr * d[c] / r;
                dE[3 * j + c] -= dedr * d[c] / r;
            }
    }
    if (grad) {
        const double* xo = x + 3 * L->origin;
        for (int c = 0; c < 6 + L->n_rot; ++c) grad[c] = 0.0;
        for (int i = 0; i < n; ++i) {
            double r[3], t[3];
            v_sub(x + 3 * i, xo, r);
            v_cross(r, dE + 3 * i, t);
            for (int c = 0; c < 3; ++c) { grad[c] += dE[3 * i + c]; grad[3 + c] += t[c]; }
        }
        for (int k = 0; k < L->n_rot; ++k) {
            double axis[3];
            v_sub(x + 3 * L->tor_c[k], x + 3 * L->tor_p[k], axis);
            double len = v_norm(axis);
            for (int c = 0; c < 3; ++c) axis[c] /= len;
            double tau[3] = {0, 0, 0};
            for (int i = 0; i < n; ++i) {
                if (!L->moves[(size_t)k * n + i]) continue;
                double r[3], t[3];
                v_sub(x + 3 * i, x + 3 * L->tor_c[k], r);
                v_cross(r, dE + 3 * i, t);
                for (int c = 0; c < 3; ++c) tau[c] += t[c];
            }
            grad[6 + k] = v_dot(axis, tau);
        }
    }
    if (parts) { parts[0] = e_inter; parts[1] = e_intra; }
    free(x); free(dE);
    return e_inter + e_intra;
}

/* Per-atom coordinates and dSF/dx (for gradient tests of the kinematics). */
double or_score_atoms(const or_ligand* L, const or_grid* G, const double* xyz, double* dEdx) {
    int n = L->n;
    double e = 0.0;
    for (int i = 0; i < 3 * n; ++i) dEdx[i] = 0.0;
    for (int i = 0; i < n; ++i) e += or_grid_eval(G, L->xs[i], xyz + 3 * i, dEdx + 3 * i);
    for (int p = 0; p < L->n_pairs; ++p) {
        int i = L->pairs[2 * p], j = L->pairs[2 * p + 1];
        double d[3], dedr;
        v_sub(xyz + 3 * i, xyz + 3 * j, d);
        double r = v_norm(d);
        e += or_pair_energy(L->xs[i], L->xs[j], r, &dedr);
        if (r > 0.0)
            for (int c = 0; c < 3; ++c) {
                dEdx[3 * i + c] += dedr * d[c] / r;
                dEdx[3 * j + c] -= dedr * d[c] / r;
            }
    }
    return e;
}

/* Tangent step: translation += s[0:3]; q <- exp(s[3:6]/2) (x) q; psi += s[6:]. */
void or_retract(int n_rot, const double* pot, const double* step, double* out) {
    if (out != pot) memcpy(out, pot, sizeof(double) * (7 + n_rot));
    for (int c = 0; c < 3; ++c) out[c] = pot[c] + step[c];
    quat_rotate_by(out + 3, step + 3);
    for (int k = 0; k < n_rot; ++k) out[7 + k] = pot[7 + k] + step[6 + k];
}

/* --------------------------------------------------------------------- RILC-BFGS --- */
typedef struct {
    int n_tan, n_state;
    double (*eval)(void* ctx, const double* state, double* grad);
    void (*retract)(void* ctx, const double* state, const double* step, double* out);
    void* ctx;
} or_problem;

typedef struct {
    int m;           /* L-BFGS memory (pairs kept) */
    int max_iter;    /* iteration budget K */
    int max_trials;  /* line-search trials per iteration */
    double rho;      /* Armijo constant, Eq. 7 */
    double sigma;    /* weak-Wolfe constant, Eq. 8 */
    double eps;      /* Eq. 11 curvature threshold and Eq. 12 gradient tolerance */
} or_bfgs_params;

#define OR_MAXN 64
#define OR_MAXM 16

/* Minimises P from state (in/out). Returns the final SF; g receives its gradient; *evals is
 * incremented per objective evaluation.
 *   d_0 = -g (Eq. 6); later d = -H g by the two-loop recursion over the m most recent stored
 *   pairs (s, y) (Eq. 10), initial scaling s.y / y.y of the newest pair;
 *   stop if g.d >= 0 (non-descent) or ||g|| <= eps (Eq. 12) or after max_iter iterations;
 *   Lewis-Overton: lambda = 1; if SF(x + lambda d) > SF(x) + lambda rho g.d (Eq. 7 as printed,
 *   the Armijo test failing) the upper bound becomes lambda; else if g_new.d < sigma g.d
 *   (Eq. 8 as printed, the weak Wolfe test failing) the lower bound becomes lambda; else the
 *   step is accepted. Next lambda: 2 lambda while no upper bound, else the midpoint. After
 *   max_trials without acceptance the largest Armijo-satisfying lambda tried is taken, or the
 *   search stops if none was;
 *   x_{k+1} = x_k + lambda d (Eq. 9); the pair is stored iff y.s / ||s||^2 > eps ||g_k|| (Eq. 11). */
double or_bfgs(const or_problem* P, const or_bfgs_params* bp, double* state, double* g, long* evals) {
    int n = P->n_tan, ns = P->n_state, m = bp->m;
    double S[OR_MAXM][OR_MAXN], Y[OR_MAXM][OR_MAXN], RH[OR_MAXM];
    int stored = 0, head = 0; /* ring buffer: newest at (head - 1) mod m */
    double x[OR_MAXN * 2], xt[OR_MAXN * 2], xlo[OR_MAXN * 2];
    double gt[OR_MAXN], glo[OR_MAXN], d[OR_MAXN], q[OR_MAXN], alpha[OR_MAXM];
    memcpy(x, state, sizeof(double) * ns);
    double f = P->eval(P->ctx, x, g);
    (*evals)++;
    for (int it = 0; it < bp->max_iter; ++it) {
        /* direction */
        for (int c = 0; c < n; ++c) q[c] = g[c];
        for (int a = 0; a < stored; ++a) {
            int j = ((head - 1 - a) % m + m) % m;
            double s = 0;
            for (int c = 0; c < n; ++c) s += S[j][c] * q[c];
            alpha[a] = RH[j] * s;
            for (int c = 0; c < n; ++c) q[c] -= alpha[a] * Y[j][c];
        }
        if (stored > 0) {
            int j = ((head - 1) % m + m) % m;
            double sy = 0, yy = 0;
            for (int c = 0; c < n; ++c) { sy += S[j][c] * Y[j][c]; yy += Y[j][c] * Y[j][c]; }
            for (int c = 0; c < n; ++c) q[c] *= sy / yy;
        }
        for (int a = stored - 1; a >= 0; --a) {
            int j = ((head - 1 - a) % m + m) % m;
            double b = 0;
            for (int c = 0; c < n; ++c) b += Y[j][c] * q[c];
            b *= RH[j];
            for (int c = 0; c < n; ++c) q[c] += S[j][c] * (alpha[a] - b);
        }
        for (int c = 0; c < n; ++c) d[c] = -q[c];
        double gd = 0;
        for (int c = 0; c < n; ++c) gd += g[c] * d[c];
        if (!(gd < 0)) break;

        /* Lewis-Overton line search */
        double lam = 1.0, lo = 0.0, hi = -1.0, flo = 0.0, ft = 0.0;
        int accepted = 0, have_lo = 0;
        for (int tr = 0; tr < bp->max_trials; ++tr) {
            double step[OR_MAXN];
            for (int c = 0; c < n; ++c) step[c] = lam * d[c];
            P->retract(P->ctx, x, step, xt);
            ft = P->eval(P->ctx, xt, gt);
            (*evals)++;
            double gtd = 0;
            for (int c = 0; c < n; ++c) gtd += gt[c] * d[c];
            if (!(ft <= f + lam * bp->rho * gd)) {          /* Eq. 7 holds: Armijo fails */
                hi = lam;
            } else if (gtd < bp->sigma * gd) {               /* Eq. 8 holds: Wolfe fails */
                lo = lam; have_lo = 1; flo = ft;
                memcpy(xlo, xt, sizeof(double) * ns);
                memcpy(glo, gt, sizeof(double) * n);
            } else {
                accepted = 1;
                break;
            }
            lam = hi < 0 ? 2.0 * lam : 0.5 * (lo + hi);
        }
        if (!accepted) {
            if (!have_lo) break;
            lam = lo; ft = flo;
            memcpy(xt, xlo, sizeof(double) * ns);
            memcpy(gt, glo, sizeof(double) * n);
        }
        /* curvature-guarded history update (Eq. 10-11) */
        double sv[OR_MAXN], yv[OR_MAXN], ys = 0, ss = 0, gn = 0;
        for (int c = 0; c < n; ++c) {
            sv[c] = lam * d[c]; yv[c] = gt[c] - g[c];
            ys += yv[c] * sv[c]; ss += sv[c] * sv[c]; gn += g[c] * g[c];
        }
        if (ss > 0 && ys / ss > bp->eps * sqrt(gn)) {
            memcpy(S[head], sv, sizeof(double) * n);
            memcpy(Y[head], yv, sizeof(double) * n);
            RH[head] = 1.0 / ys;
            head = (head + 1) % m;
            if (stored < m) stored++;
        }
        memcpy(x, xt, sizeof(double) * ns);
        memcpy(g, gt, sizeof(double) * n);
        f = ft;
        double gn1 = 0;
        for (int c = 0; c < n; ++c) gn1 += g[c] * g[c];
        if (sqrt(gn1) <= bp->eps) break;                      /* Eq. 12 */
    }
    memcpy(state, x, sizeof(double) * ns);
    return f;
}

/* ------------------------------------------------------------- docking problem glue --- */
typedef struct { const or_ligand* L; const or_grid* G; } dock_ctx;

static double dock_eval(void* c, const double* pot, double* grad) {
    dock_ctx* d = (dock_ctx*)c;
    return or_score(d->L, d->G, pot, grad, NULL);
}
static void dock_retract(void* c, const double* pot, const double* step, double* out) {
    dock_ctx* d = (dock_ctx*)c;
    or_retract(d->L->n_rot, pot, step, out);
}

/* BFGS on the docking objective from a POT (in/out); returns SF. */
double or_bfgs_pose(const or_ligand* L, const or_grid* G, const or_bfgs_params* bp, double* pot,
                    double* grad, long* evals) {
    dock_ctx c = {L, G};
    or_problem P = {6 + L->n_rot, 7 + L->n_rot, dock_eval, dock_retract, &c};
    or_bfgs_params b = *bp;
    if (b.max_iter <= 0) b.max_iter = (25 + L->n) / 3;
    double g[OR_MAXN];
    double f = or_bfgs(&P, &b, pot, g, evals);
    if (grad) memcpy(grad, g, sizeof(double) * (6 + L->n_rot));
    return f;
}

/* ------------------------------------------------------------- MC chain (Algorithm 2) --- */
typedef struct {
    uint64_t seed;
    int steps;
    double temperature;   /* Metropolis temperature (Eq. 13 reading) */
    double amplitude;     /* translation mutation radius, A */
    or_bfgs_params bfgs;  /* max_iter <= 0: floor((25 + N_atoms) / 3) */
    int focc;             /* first-order consistency check: neighbours kept (0 = off, <= 4) */
    double focc_min_delta;/* coordinates closer than this carry no sign information */
} or_mc_params;

/* Random conformation (Algorithm 2, random_conformation): draws 0-2 translation uniform in the
 * box, draws 3-5 a uniform unit quaternion (Shoemake), draws 6.. torsions in [-pi, pi). */
void or_random_conformation(const or_ligand* L, const double center[3], const double size[3],
                            uint64_t seed, uint32_t unit, uint32_t chain, double* pot) {
    or_stream s = {chain, unit, 0u, seed};
    for (int c = 0; c < 3; ++c) pot[c] = center[c] + (stream_uniform(&s, c) - 0.5) * size[c];
    double u1 = stream_uniform(&s, 3), u2 = stream_uniform(&s, 4), u3 = stream_uniform(&s, 5);
    pot[3] = sqrt(1 - u1) * sin(2 * OR_PI * u2);
    pot[4] = sqrt(1 - u1) * cos(2 * OR_PI * u2);
    pot[5] = sqrt(u1) * sin(2 * OR_PI * u3);
    pot[6] = sqrt(u1) * cos(2 * OR_PI * u3);
    for (int k = 0; k < L->n_rot; ++k) pot[7 + k] = -OR_PI + 2 * OR_PI * stream_uniform(&s, 6 + k);
}

/* Uniform point in the unit ball from three uniforms: z = 2a - 1, phi = 2 pi b, r = cbrt(c). */
static void ball_point(double a, double b, double c, double p[3]) {
    double z = 2 * a - 1, phi = 2 * OR_PI * b, r = cbrt(c);
    double s = sqrt(1 - z * z > 0 ? 1 - z * z : 0);
    p[0] = r * s * cos(phi); p[1] = r * s * sin(phi); p[2] = r * z;
}

/* Mutation R (Eq. 2) at MC step `step` (draw stream step + 1): word 0 picks one entity among
 * {position, orientation, psi_1..psi_Nrot} uniformly as floor(w * (2 + N_rot) / 2^32);
 * draws 1-3: a point p in the unit ball; position += amplitude * p, orientation rotated by
 * (amplitude / R_gyr) * p; draw 4: the chosen torsion is redrawn in [-pi, pi). */
void or_mutate(const or_ligand* L, const double* pot_in, double amplitude, uint64_t seed,
               uint32_t unit, uint32_t chain, int step, double* pot) {
    or_stream s = {chain, unit, (uint32_t)(step + 1), seed};
    memcpy(pot, pot_in, sizeof(double) * (7 + L->n_rot));
    uint32_t w = stream_word(&s, 0);
    int entity = (int)(((uint64_t)w * (uint64_t)(2 + L->n_rot)) >> 32);
    double p[3];
    ball_point(stream_uniform(&s, 1), stream_uniform(&s, 2), stream_uniform(&s, 3), p);
    if (entity == 0) {
        for (int c = 0; c < 3; ++c) pot[c] += amplitude * p[c];
    } else if (entity == 1) {
        double om[3];
        double sc = L->rgyr > 1e-9 ? amplitude / L->rgyr : 0.0;
        for (int c = 0; c < 3; ++c) om[c] = sc * p[c];
        quat_rotate_by(pot + 3, om);
    } else {
        pot[7 + (entity - 2)] = -OR_PI + 2 * OR_PI * stream_uniform(&s, 4);
    }
}

/* Metropolis draw of MC step `step` (draw 5 of its stream). */
double or_metropolis_uniform(uint64_t seed, uint32_t unit, uint32_t chain, int step) {
    or_stream s = {chain, unit, (uint32_t)(step + 1), seed};
    return stream_uniform(&s, 5);
}

/* Metropolis criterion (Eq. 13, read as a Boltzmann factor at temperature T): always accept an
 * improvement, else accept iff u < exp((e_cur - e_new) / T). */
int or_metropolis_accept(double e_cur, double e_new, double temperature, double u) {
    return (e_new < e_cur) || (u < exp((e_cur - e_new) / temperature));
}

/* ------------------------------------------- first-order consistency check (Eq. 4-5) --- */
#define OR_FOCC_MAX 4

/* Tangent-space difference a - b of two POTs: translation difference, the rotation vector w
 * with q_a = exp(w / 2) (x) q_b (shortest rotation; both quaternions normalised first), torsion
 * differences wrapped into [-pi, pi). */
void or_tangent_delta(int n_rot, const double* a, const double* b, double* out) {
    for (int c = 0; c < 3; ++c) out[c] = a[c] - b[c];
    double qa[4], qb[4], na = 0, nb = 0;
    for (int k = 0; k < 4; ++k) { na += a[3 + k] * a[3 + k]; nb += b[3 + k] * b[3 + k]; }
    na = sqrt(na); nb = sqrt(nb);
    qa[0] = a[3] / na; qb[0] = b[3] / nb;
    for (int k = 1; k < 4; ++k) { qa[k] = a[3 + k] / na; qb[k] = -b[3 + k] / nb; }   /* qb <- conj */
    double r[4];
    quat_mul(qa, qb, r);
    if (r[0] < 0) for (int k = 0; k < 4; ++k) r[k] = -r[k];
    double vn = sqrt(r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    double scale = vn > 1e-15 ? 2.0 * atan2(vn, r[0]) / vn : 2.0;
    for (int c = 0; c < 3; ++c) out[3 + c] = scale * r[1 + c];
    for (int k = 0; k < n_rot; ++k) {
        double d = a[7 + k] - b[7 + k];
        d = d - 2 * OR_PI * floor((d + OR_PI) / (2 * OR_PI));
        out[6 + k] = d;
    }
}

static int sgn(double v) { return (v > 0) - (v < 0); }

/* The check of Eq. 4-5 for a candidate C_i' (SF f_i, tangent gradient g_i) against stored
 * neighbours C_j (SF f_j, gradient g_j). Reading (the paper leaves the neighbours and the
 * quantifiers open): along a tangent coordinate p where the two differ by more than min_delta,
 * Eq. 4 (the derivative changes sign between them) or Eq. 5 (the secant slope
 * (SF_i - SF_j) / (C_i - C_j)_p disagrees in sign with the derivative at C_i') means a stationary
 * point may lie between them. The candidate passes (is worth a local search) if every neighbour
 * has such a coordinate; it fails if some neighbour has none, i.e. the candidate lies on a
 * slope that runs down to that neighbour along every coordinate and would roll back to it.
 * No neighbour: pass. Returns 1 (pass) or 0 (fail). */
int or_focc_pass(const or_ligand* L, const double* pot_i, double f_i, const double* g_i, int n_nb,
                 const double* pots, const double* fs, const double* gs, double min_delta) {
    int n_rot = L->n_rot, n_tan = 6 + n_rot, np = 7 + n_rot;
    for (int j = 0; j < n_nb; ++j) {
        double dl[OR_MAXN];
        or_tangent_delta(n_rot, pot_i, pots + (size_t)j * np, dl);
        int evidence = 0;
        for (int p = 0; p < n_tan && !evidence; ++p) {
            if (!(fabs(dl[p]) > min_delta)) continue;
            int gi = sgn(g_i[p]), gj = sgn(gs[(size_t)j * n_tan + p]);
            if (gi * gj <= 0) evidence = 1;                                   /* Eq. 4 */
            else if (gi * sgn((f_i - fs[j]) * dl[p]) <= 0) evidence = 1;      /* Eq. 5 */
        }
        if (!evidence) return 0;
    }
    return 1;
}

/* The last H current conformations of a chain with SF and gradient (the neighbours of Eq. 4-5),
 * stored contiguously in push order modulo H. */
typedef struct {
    int H, n, head, np, n_tan;
    double pot[OR_FOCC_MAX * OR_MAXN * 2], g[OR_FOCC_MAX * OR_MAXN], f[OR_FOCC_MAX];
} focc_ring;

static void focc_push(focc_ring* r, const double* pot, const double* g, double f) {
    if (r->H == 0) return;
    memcpy(r->pot + (size_t)r->head * r->np, pot, sizeof(double) * r->np);
    memcpy(r->g + (size_t)r->head * r->n_tan, g, sizeof(double) * r->n_tan);
    r->f[r->head] = f;
    r->head = (r->head + 1) % r->H;
    if (r->n < r->H) r->n++;
}

/* One chain of Algorithm 2: start C_cur = C_best = random conformation; each step mutate,
 * optimise (RILC-BFGS), accept with p = min(1, exp((e_cur - e_new) / T)); an accepted candidate
 * that beats the best is refined by a second RILC-BFGS run and becomes both the current and the
 * best conformation. With the first-order consistency check on (focc > 0), each mutated candidate
 * is first evaluated with its gradient and checked (Eq. 4-5, or_focc_pass) against the chain's
 * last `focc` current conformations (the start and every accepted or refined one, with SF and
 * gradient); a candidate that fails skips the local search and enters the Metropolis test with
 * its own SF. Outputs the chain's best POT and SF, and its evaluation count. */
void or_mc_chain(const or_ligand* L, const or_grid* G, const double center[3], const double size[3],
                 const or_mc_params* mp, uint32_t unit, uint32_t chain, double* best_pot,
                 double* best_e, long* evals) {
    int np = 7 + L->n_rot, n_tan = 6 + L->n_rot;
    or_bfgs_params bp = mp->bfgs;
    if (bp.max_iter <= 0) bp.max_iter = (25 + L->n) / 3;
    double cur[OR_MAXN * 2], cand[OR_MAXN * 2], best[OR_MAXN * 2];
    double g_cur[OR_MAXN], g_cand[OR_MAXN];
    focc_ring nb;
    nb.H = mp->focc < 0 ? 0 : (mp->focc > OR_FOCC_MAX ? OR_FOCC_MAX : mp->focc);
    nb.n = 0; nb.head = 0; nb.np = np; nb.n_tan = n_tan;
    long ev = 0;
    or_random_conformation(L, center, size, mp->seed, unit, chain, cur);
    double e_cur = or_score(L, G, cur, nb.H ? g_cur : NULL, NULL);
    ev++;
    memcpy(best, cur, sizeof(double) * np);
    double e_best = e_cur;
    focc_push(&nb, cur, g_cur, e_cur);
    for (int st = 0; st < mp->steps; ++st) {
        or_mutate(L, cur, mp->amplitude, mp->seed, unit, chain, st, cand);
        double e_new;
        int optimise = 1;
        if (nb.H) {
            e_new = or_score(L, G, cand, g_cand, NULL);
            ev++;
            optimise = or_focc_pass(L, cand, e_new, g_cand, nb.n, nb.pot, nb.f, nb.g, mp->focc_min_delta);
        }
        if (optimise) e_new = or_bfgs_pose(L, G, &bp, cand, g_cand, &ev);
        double u = or_metropolis_uniform(mp->seed, unit, chain, st);
        if (or_metropolis_accept(e_cur, e_new, mp->temperature, u)) {
            memcpy(cur, cand, sizeof(double) * np);
            memcpy(g_cur, g_cand, sizeof(double) * n_tan);
            e_cur = e_new;
            if (e_cur < e_best) {
                e_cur = or_bfgs_pose(L, G, &bp, cur, g_cur, &ev);
                memcpy(best, cur, sizeof(double) * np);
                e_best = e_cur;
            }
            focc_push(&nb, cur, g_cur, e_cur);
        }
    }
    memcpy(best_pot, best, sizeof(double) * np);
    *best_e = e_best;
    *evals = ev;
}

/* All chains of one (ligand, pocket) unit; OpenMP over independent chains. */
void or_mc_chains(const or_ligand* L, const or_grid* G, const double center[3], const double size[3],
                  const or_mc_params* mp, uint32_t unit, int n_chains, double* best_pot,
                  double* best_e, long* evals, int n_threads) {
    int np = 7 + L->n_rot;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < n_chains; ++c)
        or_mc_chain(L, G, center, size, mp, unit, (uint32_t)c, best_pot + (size_t)c * np,
                    best_e + c, evals + c);
    (void)n_threads;
}

/* ------------------------------------------------- rescoring of selected poses (Alg. 2) --- */
/* e_inter of a posed ligand (atom coordinates in input order) summed directly over the receptor
 * atoms: sum_i sum_j E(type_i, type_j, |x_i - x_j|) with the 8 A cutoff; no grid, no box. */
double or_direct_inter(const or_ligand* L, int n_rec, const double* rec_xyz, const int32_t* rec_types,
                       const double* lig_xyz) {
    double e = 0.0;
    for (int i = 0; i < L->n; ++i)
        for (int j = 0; j < n_rec; ++j) {
            double d[3];
            v_sub(lig_xyz + 3 * i, rec_xyz + 3 * j, d);
            e += or_pair_energy(L->xs[i], rec_types[j], v_norm(d), NULL);
        }
    return e;
}

/* ------------------------------------------------------- top-k selection (Algorithm 2) --- */
/* Sort candidates by SF ascending (ties: lower index first), keep a candidate if its RMSD to
 * every kept one (fixed atom correspondence) is >= rmsd_min, stop at k. Returns the count. */
int or_topk(int n_cand, const double* score, const double* xyz, int n_atoms, int k,
            double rmsd_min, int32_t* out) {
    int* idx = (int*)malloc(sizeof(int) * (n_cand ? n_cand : 1));
    for (int i = 0; i < n_cand; ++i) idx[i] = i;
    for (int a = 1; a < n_cand; ++a) { /* stable insertion sort */
        int v = idx[a], j = a - 1;
        while (j >= 0 && score[idx[j]] > score[v]) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = v;
    }
    int kept = 0;
    for (int a = 0; a < n_cand && kept < k; ++a) {
        int c = idx[a], ok = 1;
        for (int b = 0; b < kept && ok; ++b) {
            double s = 0;
            for (int i = 0; i < 3 * n_atoms; ++i) {
                double d = xyz[(size_t)c * 3 * n_atoms + i] - xyz[(size_t)out[b] * 3 * n_atoms + i];
                s += d * d;
            }
            if (sqrt(s / n_atoms) < rmsd_min) ok = 0;
        }
        if (ok) out[kept++] = c;
    }
    free(idx);
    return kept;
}

/* Vina-style reported affinity of a pose: e_inter / (1 + w_rot N_rot). */
double or_affinity(double e_inter, int n_rot) { return e_inter / (1.0 + W_ROT * n_rot); }
