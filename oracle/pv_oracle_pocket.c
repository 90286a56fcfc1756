/*
 * pv_oracle_pocket.c -- plain, slow, FP64 CPU oracle for the pocket-side steps of PocketVina
 * (Methods "Pocket Prediction with P2Rank", Eq. 1-2, Supplementary Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, call or execute this file;
 * only the test suite, the smoke check and the CPU-baseline leg of the benchmark do. It shares
 * no code, header, table or constant with the CUDA implementation.
 *
 * What it computes, in the order of Supplementary Algorithm 1:
 *   Step 1  solvent-accessible surface (SAS) points. The paper names a numerical surface
 *           algorithm without its parameters; this is the numerical SAS of Shrake & Rupley
 *           (J. Mol. Biol. 79, 1973): every atom i carries n_s points on its expanded sphere of
 *           radius a_i = R_i + probe, and a point is kept unless it lies strictly inside the
 *           expanded sphere of another atom (|p - x_j| < a_j). The n_s directions are the
 *           spherical Fibonacci lattice (Gonzalez, Math. Geosci. 42, 2010): for k = 0 .. n_s-1,
 *           z_k = 1 - (2k + 1) / n_s, azimuth k * pi * (3 - sqrt 5).
 *   Step 2  Eq. 1 feature sums at given points: f_p^phi = sum over atoms a of
 *           max(0, 1 - |x_a - p| / r_feat) * phi(a), r_feat = 6 A; protrusion = the number of
 *           atoms with |x_a - p| <= r_prot, r_prot = 10 A.
 *   Step 3  the Random Forest score s_p is an input (no trained model is part of this build).
 *   Step 4  points with s_p >= theta (the algorithm's comparison) joined by single linkage:
 *           two points are in one cluster iff a chain of points links them with every hop
 *           <= link (3 A).
 *   Step 5  per cluster: Eq. 2 score S_K = sum of s_p^2, centre = mean of its points, size;
 *           clusters sorted by S_K descending, ties by the lowest point index.
 * Every routine below is brute force over all atom or point pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OP_PI 3.14159265358979323846

/* Spherical Fibonacci lattice: n unit vectors, row-major [n][3]. */
void or_sphere_lattice(int n, double* dirs) {
    const double golden_angle = OP_PI * (3.0 - sqrt(5.0));
    for (int k = 0; k < n; ++k) {
        const double z = 1.0 - (2.0 * k + 1.0) / n;
        const double rho = sqrt(fmax(0.0, 1.0 - z * z));
        const double phi = golden_angle * k;
        dirs[3 * k + 0] = rho * cos(phi);
        dirs[3 * k + 1] = rho * sin(phi);
        dirs[3 * k + 2] = z;
    }
}

/* Step 1 for the atoms listed in sel[0 .. n_sel-1] (sel == NULL: every atom, in order).
 * Row s*n_s + k of the outputs belongs to atom sel[s], lattice direction k:
 *   pts    [..][3]  x_i + a_i * u_k
 *   keep   [..]     1 if the point is on the SAS, else 0
 *   margin [..]     min over j != i of (|p - x_j| - a_j): negative iff buried; 1e300 if n == 1.
 * radius[i] = R_i (vdW radius); a_i = R_i + probe. */
void or_sas_points(int n_atoms, const double* xyz, const double* radius, double probe, int n_s,
                   int n_sel, const int32_t* sel, uint8_t* keep, double* pts, double* margin) {
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)(n_s > 0 ? n_s : 1));
    or_sphere_lattice(n_s, dirs);
    const int rows = sel ? n_sel : n_atoms;
#pragma omp parallel for schedule(dynamic, 4)
    for (int s = 0; s < rows; ++s) {
        const int i = sel ? sel[s] : s;
        const double ai = radius[i] + probe;
        for (int k = 0; k < n_s; ++k) {
            const size_t row = (size_t)s * n_s + k;
            double p[3];
            for (int c = 0; c < 3; ++c) p[c] = xyz[3 * i + c] + ai * dirs[3 * k + c];
            double m = 1e300;
            for (int j = 0; j < n_atoms; ++j) {
                if (j == i) continue;
                const double dx = p[0] - xyz[3 * j], dy = p[1] - xyz[3 * j + 1], dz = p[2] - xyz[3 * j + 2];
                const double gap = sqrt(dx * dx + dy * dy + dz * dz) - (radius[j] + probe);
                if (gap < m) m = gap;
            }
            memcpy(pts + 3 * row, p, sizeof(p));
            margin[row] = m;
            keep[row] = m >= 0.0;
        }
    }
    free(dirs);
}

/* Step 2 (Eq. 1 and the protrusion count) at n_pts given points.
 * props [n_atoms][n_props]; feat [n_pts][n_props]; protrusion [n_pts]. */
void or_point_features(int n_atoms, const double* xyz, int n_props, const double* props, int n_pts,
                       const double* pts, double r_feat, double r_prot, double* feat,
                       int32_t* protrusion) {
#pragma omp parallel for schedule(static)
    for (int p = 0; p < n_pts; ++p) {
        double* f = feat + (size_t)p * n_props;
        for (int q = 0; q < n_props; ++q) f[q] = 0.0;
        int32_t count = 0;
        for (int a = 0; a < n_atoms; ++a) {
            const double dx = xyz[3 * a] - pts[3 * p], dy = xyz[3 * a + 1] - pts[3 * p + 1],
                         dz = xyz[3 * a + 2] - pts[3 * p + 2];
            const double d = sqrt(dx * dx + dy * dy + dz * dz);
            const double w = fmax(0.0, 1.0 - d / r_feat);
            for (int q = 0; q < n_props; ++q) f[q] += w * props[(size_t)a * n_props + q];
            if (d <= r_prot) ++count;
        }
        protrusion[p] = count;
    }
}

static int uf_root(int32_t* parent, int x) {
    while (parent[x] != x) x = parent[x];
    return x;
}

/* Steps 4-5. Returns the number of clusters K. Outputs (each sized for n, first K rows used):
 *   root[i]    the lowest point index of i's cluster, -1 if s_i < theta (or s_i is NaN)
 *   cluster[i] the rank of i's cluster (0 = highest S_K), -1 if below the threshold
 *   c_score[r] S_K, c_center[r][3] mean of the points, c_size[r], c_first[r] lowest index. */
int or_cluster_points(int n, const double* pts, const double* score, double theta, double link,
                      int32_t* root, int32_t* cluster, double* c_score, double* c_center,
                      int32_t* c_size, int32_t* c_first) {
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) parent[i] = i;
    for (int i = 0; i < n; ++i) {
        if (!(score[i] >= theta)) continue;
        for (int j = i + 1; j < n; ++j) {
            if (!(score[j] >= theta)) continue;
            const double dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1],
                         dz = pts[3 * i + 2] - pts[3 * j + 2];
            if (sqrt(dx * dx + dy * dy + dz * dz) > link) continue;
            const int ri = uf_root(parent, i), rj = uf_root(parent, j);
            if (ri < rj) parent[rj] = ri;
            else if (rj < ri) parent[ri] = rj;
        }
    }
    /* clusters in order of their lowest index, then sorted by score */
    int32_t* id_of_root = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int k = 0;
    for (int i = 0; i < n; ++i) {
        id_of_root[i] = -1;
        root[i] = score[i] >= theta ? uf_root(parent, i) : -1;
        if (root[i] == i) id_of_root[i] = k++;
    }
    double* s = (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
    double* c = (double*)calloc((size_t)(k > 0 ? k : 1) * 3, sizeof(double));
    int32_t* sz = (int32_t*)calloc((size_t)(k > 0 ? k : 1), sizeof(int32_t));
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    for (int i = 0; i < n; ++i) {
        if (root[i] < 0) continue;
        const int id = id_of_root[root[i]];
        s[id] += score[i] * score[i];
        for (int a = 0; a < 3; ++a) c[3 * id + a] += pts[3 * i + a];
        sz[id] += 1;
        if (root[i] == i) first[id] = i;
    }
    /* rank: the number of clusters that sort before this one */
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    for (int a = 0; a < k; ++a) {
        int r = 0;
        for (int b = 0; b < k; ++b)
            if (s[b] > s[a] || (s[b] == s[a] && first[b] < first[a])) ++r;
        rank[a] = r;
    }
    for (int a = 0; a < k; ++a) {
        const int r = rank[a];
        c_score[r] = s[a];
        for (int d = 0; d < 3; ++d) c_center[3 * r + d] = c[3 * a + d] / sz[a];
        c_size[r] = sz[a];
        c_first[r] = first[a];
    }
    for (int i = 0; i < n; ++i) cluster[i] = root[i] < 0 ? -1 : rank[id_of_root[root[i]]];
    free(parent); free(id_of_root); free(s); free(c); free(sz); free(first); free(rank);
    return k;
}
