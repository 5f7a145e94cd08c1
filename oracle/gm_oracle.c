/*
 * gm_oracle.c -- plain FP64 CPU oracle of the Gaussian Moment Neural Network (GMNN)
 * energy, forces, virial and force-matching parameter gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library calls, links or includes this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code with the CUDA path.  Compile with -ffp-contract=off so that every
 * floating-point operation rounds exactly as written (the neighbour-membership rule is
 * compared bit for bit against the GPU).
 *
 * What it computes (section "Machine Learning Interatomic Potentials" of the paper):
 *   E(S)       = sum_i E_i                                        (Eq. energy_sum)
 *   Psi_{i,L,s}= sum_{j != i} R_{Zi,Zj,s}(r_ij) rhat_ij^{(x)L}, L=0..3 (Eq. basis_fn)
 *   G_i        = full tensor contractions of Psi up to L=3           (Eq. contraction)
 *   E_i        = sigma_{Zi} NN(G_i) + mu_{Zi}                       (Eq. scale_shift)
 *   F          = -dE/dr, virial W = -dE/d(strain)   (Software Architecture, Model
 *                                                    Abstractions: forces and virials
 *                                                    as gradients)
 * Readings where the paper is silent (the paper prints neither the basis formula nor
 * the complete contraction list):
 *   Phi_k(r) = exp(-gamma (r - mu_k)^2), mu_k = r_min + k (r_c - r_min)/(n_b - 1),
 *              gamma = n_b^2 / r_c^2                      ("equidistant Gaussians")
 *   or, as the alternative basis, the Bessel-like functions of Kocer et al.
 *   f_k(r)   = a_k [j0((k+1) pi r/r_c) + j0((k+2) pi r/r_c)]   (see basis_eval)
 *   f_c(r)   = (cos(pi r / r_c) + 1) / 2 for r < r_c, else 0
 *   R_s(r)   = f_c(r) n_b^{-1/2} sum_k beta[Zi][Zj][s][k] Phi_k(r)  (ordered pair)
 *   features = 8 families (#1 Psi0; #2 Psi1.Psi1; #3 Psi2:Psi2; #4 Psi3:Psi3;
 *              #5 tr(Psi2 Psi2 Psi2); #6 Psi1 Psi2 Psi1; #7 Psi3 Psi3 Psi2 (two shared
 *              indices); #8 Psi1 Psi3 Psi2), with the radial-index symmetries removed;
 *              360 features for n_r = 5.  #2 and #8 are the two printed in the paper.
 *   NN       = w3 . phi(W2^T phi(W1^T G + b1) + b2) + b3, phi = tanh or SiLU
 *   loss     = (wE/B) sum_b ((E_b - E_b^ref)/N_b)^2 + (wF/(3N)) sum_i |F_i - F_i^ref|^2
 * Neighbour rule: pairs (i, j, n) with |r'_j - r'_i + n.cell| < r_c, excluding only
 * (j == i, n == 0); periodic self-images are kept.  r' are positions wrapped into the
 * cell by the rule in wrap_axis(); the reported shift is relative to the caller's
 * (unwrapped) positions.
 *
 * Parity status: every function here is pinned by the CPU tests (finite differences,
 * invariances, closed forms of the dimer and of axis-aligned configurations, trace
 * identities, brute force, and an independent autograd restatement).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXR 8            /* maximum number of radial functions */
#define OR_NT(nr) (40 * (nr)) /* full-tensor state per atom: (1+3+9+27) per radial fn */

typedef struct {
    int n_species, n_basis, n_radial, n_hidden, activation; /* 0 = tanh, 1 = SiLU */
    double r_min, r_cut;
    const double *beta;  /* [S][S][n_radial][n_basis] */
    const double *W1;    /* [F][H] */
    const double *b1;    /* [H] */
    const double *W2;    /* [H][H] */
    const double *b2;    /* [H] */
    const double *w3;    /* [H] */
    const double *b3;    /* [1] */
    const double *sigma; /* [S] */
    const double *mu;    /* [S] */
    int basis;           /* 0: equidistant Gaussians, 1: Bessel-like functions (Kocer et al.) */
} or_model;

typedef struct { /* parameter gradient, same shapes as or_model */
    double *beta, *W1, *b1, *W2, *b2, *w3, *b3, *sigma, *mu;
} or_grad;

/* ------------------------------------------------------------------ neighbours */

/* Wrap one Cartesian coordinate of an orthorhombic cell of edge L into [0, L).
 * Returns the wrapped value and the image count m with x' = x - m L.  The GPU library
 * applies the identical sequence of correctly rounded operations. */
static double wrap_axis(double x, double L, int *m_out) {
    double m = floor(x / L);
    double xw = x - m * L;
    if (xw < 0.0) { m -= 1.0; xw = x - m * L; }
    if (xw >= L) { m += 1.0; xw = x - m * L; }
    if (xw < 0.0 || xw >= L) xw = 0.0;
    *m_out = (int)m;
    return xw;
}

static int is_orthorhombic(const double *c) {
    return c[1] == 0.0 && c[2] == 0.0 && c[3] == 0.0 && c[5] == 0.0 && c[6] == 0.0 && c[7] == 0.0;
}

static void inv3(const double *a, double *inv) { /* inverse of row-major 3x3 */
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                 a[2] * (a[3] * a[7] - a[4] * a[6]);
    inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

/* Wrap all atoms of one structure.  xw[3n], m[3n]. */
static void wrap_structure(int n, const double *pos, const double *cell, const unsigned char *pbc,
                           double *xw, int *m) {
    if (is_orthorhombic(cell)) {
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                if (pbc[a]) xw[3 * i + a] = wrap_axis(pos[3 * i + a], cell[4 * a], &m[3 * i + a]);
                else { xw[3 * i + a] = pos[3 * i + a]; m[3 * i + a] = 0; }
            }
        return;
    }
    double inv[9];
    inv3(cell, inv);
    for (int i = 0; i < n; ++i) {
        double f[3];
        for (int a = 0; a < 3; ++a) /* fractional f = x . inv(cell) (cell rows = vectors) */
            f[a] = pos[3 * i] * inv[a] + pos[3 * i + 1] * inv[3 + a] + pos[3 * i + 2] * inv[6 + a];
        for (int a = 0; a < 3; ++a) m[3 * i + a] = pbc[a] ? (int)floor(f[a]) : 0;
        for (int c = 0; c < 3; ++c)
            xw[3 * i + c] = pos[3 * i + c] - (m[3 * i] * cell[c] + m[3 * i + 1] * cell[3 + c] +
                                              m[3 * i + 2] * cell[6 + c]);
    }
}

/* Brute-force neighbour list of a batch.  Pairs are written grouped by centre atom i
 * (global indices), so that row_ptr can be formed by counting.  Returns 0 on success,
 * 1 when more than cap pairs exist (n_pairs then holds the required count). */
static int neighbors_impl(int n_struct, const int *atom_ptr, const double *pos, const double *cell,
                          const unsigned char *pbc, double r_cut, const unsigned char *want_row, int64_t cap,
                          int *pi, int *pj, int *pshift, int64_t *n_pairs);

int or_neighbors(int n_struct, const int *atom_ptr, const double *pos, const double *cell,
                 const unsigned char *pbc, double r_cut, int64_t cap, int *pi, int *pj, int *pshift,
                 int64_t *n_pairs) {
    return neighbors_impl(n_struct, atom_ptr, pos, cell, pbc, r_cut, NULL, cap, pi, pj, pshift, n_pairs);
}

/* Rows of the same neighbour list for the centre atoms listed in rows[] only (same rule,
 * same arithmetic); used to check large systems on sampled atoms. */
int or_neighbor_rows(int n_struct, const int *atom_ptr, const double *pos, const double *cell,
                     const unsigned char *pbc, double r_cut, int n_rows, const int *rows, int64_t cap, int *pi,
                     int *pj, int *pshift, int64_t *n_pairs) {
    const int N = atom_ptr[n_struct];
    unsigned char *want = (unsigned char *)calloc(N ? N : 1, 1);
    for (int q = 0; q < n_rows; ++q) want[rows[q]] = 1;
    int rc = neighbors_impl(n_struct, atom_ptr, pos, cell, pbc, r_cut, want, cap, pi, pj, pshift, n_pairs);
    free(want);
    return rc;
}

/* All pairs (i, j, n) of centre atom i (local index within its structure) by brute force
 * over every atom j and every image n within the range nmax.  With out_j == NULL only
 * counts; else writes the pairs in the order j, then n0, n1, n2. */
static int64_t row_pairs(int i, int n, const double *xw, const int *m, const double *C, int ortho,
                         const int *nmax, double rc2, int a0, int *out_i, int *out_j, int *out_shift) {
    int64_t np = 0;
    for (int j = 0; j < n; ++j)
        for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
            for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                    if (i == j && n0 == 0 && n1 == 0 && n2 == 0) continue;
                    double d[3];
                    if (ortho) {
                        d[0] = (xw[3 * j] - xw[3 * i]) + (double)n0 * C[0];
                        d[1] = (xw[3 * j + 1] - xw[3 * i + 1]) + (double)n1 * C[4];
                        d[2] = (xw[3 * j + 2] - xw[3 * i + 2]) + (double)n2 * C[8];
                    } else {
                        for (int c = 0; c < 3; ++c)
                            d[c] = (xw[3 * j + c] - xw[3 * i + c]) + (n0 * C[c] + n1 * C[3 + c] + n2 * C[6 + c]);
                    }
                    double r2 = d[0] * d[0] + d[1] * d[1];
                    r2 = r2 + d[2] * d[2];
                    if (!(r2 < rc2)) continue;
                    if (out_j) {
                        out_i[np] = a0 + i;
                        out_j[np] = a0 + j;
                        out_shift[3 * np + 0] = n0 - m[3 * j + 0] + m[3 * i + 0];
                        out_shift[3 * np + 1] = n1 - m[3 * j + 1] + m[3 * i + 1];
                        out_shift[3 * np + 2] = n2 - m[3 * j + 2] + m[3 * i + 2];
                    }
                    ++np;
                }
    return np;
}

/* The rows are independent, so they are searched in parallel over centre atoms: a counting
 * pass, a prefix sum over the rows (in atom order), then a filling pass that writes every
 * row at its offset.  The arithmetic of each pair test is the same in both passes. */
static int neighbors_impl(int n_struct, const int *atom_ptr, const double *pos, const double *cell,
                          const unsigned char *pbc, double r_cut, const unsigned char *want_row, int64_t cap,
                          int *pi, int *pj, int *pshift, int64_t *n_pairs) {
    int64_t np = 0;
    const double rc2 = r_cut * r_cut;
    for (int b = 0; b < n_struct; ++b) {
        const int a0 = atom_ptr[b], n = atom_ptr[b + 1] - a0;
        const double *C = cell + 9 * b;
        const unsigned char *pb = pbc + 3 * b;
        double *xw = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
        int *m = (int *)malloc(sizeof(int) * 3 * (n ? n : 1));
        int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        wrap_structure(n, pos + 3 * a0, C, pb, xw, m);
        /* image range: perpendicular widths w_a = V / |b x c| etc. */
        int nmax[3];
        double vol = fabs(C[0] * (C[4] * C[8] - C[5] * C[7]) - C[1] * (C[3] * C[8] - C[5] * C[6]) +
                          C[2] * (C[3] * C[7] - C[4] * C[6]));
        for (int a = 0; a < 3; ++a) {
            const double *u = C + 3 * ((a + 1) % 3), *v = C + 3 * ((a + 2) % 3);
            double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
            double w = vol / sqrt(cx * cx + cy * cy + cz * cz);
            nmax[a] = pb[a] ? (int)ceil(r_cut / w) + 1 : 0;
        }
        const int ortho = is_orthorhombic(C);
#pragma omp parallel for schedule(dynamic, 16)
        for (int i = 0; i < n; ++i) {
            if (want_row && !want_row[a0 + i]) continue;
            cnt[i + 1] = row_pairs(i, n, xw, m, C, ortho, nmax, rc2, a0, NULL, NULL, NULL);
        }
        for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
        if (np + cnt[n] <= cap) {
#pragma omp parallel for schedule(dynamic, 16)
            for (int i = 0; i < n; ++i) {
                if (want_row && !want_row[a0 + i]) continue;
                const int64_t o = np + cnt[i];
                row_pairs(i, n, xw, m, C, ortho, nmax, rc2, a0, pi + o, pj + o, pshift + 3 * o);
            }
        }
        np += cnt[n];
        free(cnt);
        free(xw);
        free(m);
    }
    *n_pairs = np;
    return np > cap ? 1 : 0;
}

/* ------------------------------------------------------------------ radial part */

typedef struct {
    double r, u[3];
    double B[16], dB[16]; /* f_c Phi_k and its r-derivative */
} pair_basis;

static void basis_eval(const or_model *M, double r, pair_basis *pb) {
    const int nb = M->n_basis;
    const double rc = M->r_cut;
    const double gamma = (double)(nb * nb) / (rc * rc);
    double fc = 0.0, dfc = 0.0;
    if (r < rc) {
        fc = 0.5 * (cos(M_PI * r / rc) + 1.0);
        dfc = -0.5 * M_PI / rc * sin(M_PI * r / rc);
    }
    if (M->basis == 1) {
        /* Bessel-like functions of Kocer et al. (the second basis named in section "Machine
         * Learning Interatomic Potentials"): sums of two consecutive zeroth-order spherical
         * Bessel functions j0(x) = sin(x)/x whose zeros sit at r_cut,
         *   f_k(r) = a_k [j0((k+1) pi r / r_c) + j0((k+2) pi r / r_c)],
         *   a_k    = (-1)^k sqrt(2) pi r_c^(-3/2) (k+1)(k+2) / sqrt((k+1)^2 + (k+2)^2),
         * so that f_k and f_k' vanish at r_c and int_0^rc f_k^2 r^2 dr = 1; read here with the
         * same cosine cutoff and n_b^(-1/2) normalisation as the Gaussians.
         * d/dr j0(c r) = (cos(c r) - j0(c r)) / r. */
        for (int k = 0; k < nb; ++k) {
            const double n1 = k + 1.0, n2 = k + 2.0;
            const double a = ((k & 1) ? -1.0 : 1.0) * sqrt(2.0) * M_PI / pow(rc, 1.5) * n1 * n2 /
                             sqrt(n1 * n1 + n2 * n2);
            const double x1 = n1 * M_PI * r / rc, x2 = n2 * M_PI * r / rc;
            const double j1 = sin(x1) / x1, j2 = sin(x2) / x2;
            const double phi = a * (j1 + j2);
            const double dphi = a * ((cos(x1) - j1) / r + (cos(x2) - j2) / r);
            pb->B[k] = fc * phi;
            pb->dB[k] = dfc * phi + fc * dphi;
        }
        return;
    }
    for (int k = 0; k < nb; ++k) {
        double muk = M->r_min + k * (rc - M->r_min) / (nb - 1);
        double phi = exp(-gamma * (r - muk) * (r - muk));
        double dphi = -2.0 * gamma * (r - muk) * phi;
        pb->B[k] = fc * phi;
        pb->dB[k] = dfc * phi + fc * dphi;
    }
}

/* ------------------------------------------------------------------ tensors */

/* Offsets into the per-atom full-tensor state T[OR_NT(nr)]:
 *   rank 0: s                      rank 1: nr + 3 s + a
 *   rank 2: 4 nr + 9 s + 3a + b    rank 3: 13 nr + 27 s + 9a + 3b + c            */
static int toff(int nr, int L, int s) {
    switch (L) {
    case 0: return s;
    case 1: return nr + 3 * s;
    case 2: return 4 * nr + 9 * s;
    default: return 13 * nr + 27 * s;
    }
}
static const int TSIZE[4] = {1, 3, 9, 27};

/* full-tensor monomials Y_L[idx] = prod u, and their derivatives dY/dd_b */
static void monomials(const double *u, double r, double Y[4][27], double dY[4][27][3]) {
    Y[0][0] = 1.0;
    for (int b = 0; b < 3; ++b) dY[0][0][b] = 0.0;
    for (int a = 0; a < 3; ++a) {
        Y[1][a] = u[a];
        for (int b = 0; b < 3; ++b) dY[1][a][b] = ((a == b) - u[a] * u[b]) / r;
    }
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            int idx = 3 * a + c;
            Y[2][idx] = u[a] * u[c];
            for (int b = 0; b < 3; ++b)
                dY[2][idx][b] = ((a == b) - u[a] * u[b]) / r * u[c] + u[a] * ((c == b) - u[c] * u[b]) / r;
        }
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
            for (int e = 0; e < 3; ++e) {
                int idx = 9 * a + 3 * c + e;
                Y[3][idx] = u[a] * u[c] * u[e];
                for (int b = 0; b < 3; ++b)
                    dY[3][idx][b] = ((a == b) - u[a] * u[b]) / r * u[c] * u[e] +
                                    u[a] * ((c == b) - u[c] * u[b]) / r * u[e] +
                                    u[a] * u[c] * ((e == b) - u[e] * u[b]) / r;
            }
}

/* ------------------------------------------------------------------ contractions */
/* Each family is a multilinear form of 1..3 tensors.  fam_val returns its value;
 * fam_grad adds w * d(value)/d(slot k) into g[k] (g[k] may be NULL). */

static double fam_val(int fam, const double *A, const double *B, const double *C) {
    double v = 0.0;
    switch (fam) {
    case 1: return A[0];
    case 2: for (int a = 0; a < 3; ++a) v += A[a] * B[a]; return v;
    case 3: for (int a = 0; a < 9; ++a) v += A[a] * B[a]; return v;
    case 4: for (int a = 0; a < 27; ++a) v += A[a] * B[a]; return v;
    case 5: /* A_ab B_bc C_ca */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
            v += A[3 * a + b] * B[3 * b + c] * C[3 * c + a];
        return v;
    case 6: /* A_a B_ab C_b */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) v += A[a] * B[3 * a + b] * C[b];
        return v;
    case 7: /* A_abc B_abd C_cd */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) for (int d = 0; d < 3; ++d)
                v += A[9 * a + 3 * b + c] * B[9 * a + 3 * b + d] * C[3 * c + d];
        return v;
    case 8: /* A_a B_abc C_bc */
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c)
            v += A[a] * B[9 * a + 3 * b + c] * C[3 * b + c];
        return v;
    }
    return 0.0;
}

static void fam_grad(int fam, const double *A, const double *B, const double *C, double w,
                     double *gA, double *gB, double *gC) {
    switch (fam) {
    case 1: if (gA) gA[0] += w; return;
    case 2: for (int a = 0; a < 3; ++a) { if (gA) gA[a] += w * B[a]; if (gB) gB[a] += w * A[a]; } return;
    case 3: for (int a = 0; a < 9; ++a) { if (gA) gA[a] += w * B[a]; if (gB) gB[a] += w * A[a]; } return;
    case 4: for (int a = 0; a < 27; ++a) { if (gA) gA[a] += w * B[a]; if (gB) gB[a] += w * A[a]; } return;
    case 5:
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
            if (gA) gA[3 * a + b] += w * B[3 * b + c] * C[3 * c + a];
            if (gB) gB[3 * b + c] += w * A[3 * a + b] * C[3 * c + a];
            if (gC) gC[3 * c + a] += w * A[3 * a + b] * B[3 * b + c];
        }
        return;
    case 6:
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
            if (gA) gA[a] += w * B[3 * a + b] * C[b];
            if (gB) gB[3 * a + b] += w * A[a] * C[b];
            if (gC) gC[b] += w * A[a] * B[3 * a + b];
        }
        return;
    case 7:
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) for (int d = 0; d < 3; ++d) {
                if (gA) gA[9 * a + 3 * b + c] += w * B[9 * a + 3 * b + d] * C[3 * c + d];
                if (gB) gB[9 * a + 3 * b + d] += w * A[9 * a + 3 * b + c] * C[3 * c + d];
                if (gC) gC[3 * c + d] += w * A[9 * a + 3 * b + c] * B[9 * a + 3 * b + d];
            }
        return;
    case 8:
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) for (int c = 0; c < 3; ++c) {
            if (gA) gA[a] += w * B[9 * a + 3 * b + c] * C[3 * b + c];
            if (gB) gB[9 * a + 3 * b + c] += w * A[a] * C[3 * b + c];
            if (gC) gC[3 * b + c] += w * A[a] * B[9 * a + 3 * b + c];
        }
        return;
    }
}

static const int FAM_ARITY[9] = {0, 1, 2, 2, 2, 3, 3, 3, 3};
static const int FAM_RANKS[9][3] = {{0}, {0}, {1, 1}, {2, 2}, {3, 3}, {2, 2, 2}, {1, 2, 1}, {3, 3, 2}, {1, 3, 2}};

typedef struct { int fam, off[3]; } feature;

/* Feature table: family-major, then lexicographic (s1, s2, s3) under each family's
 * radial-index restriction.  Returns the number of features. */
int or_feature_table(int nr, int *fam_out, int *off_out) {
    int n = 0;
#define EMIT(F, s1, s2, s3)                                                               \
    do {                                                                                  \
        if (fam_out) {                                                                    \
            fam_out[n] = F;                                                               \
            int ss[3] = {s1, s2, s3};                                                     \
            for (int q = 0; q < 3; ++q)                                                   \
                off_out[3 * n + q] = q < FAM_ARITY[F] ? toff(nr, FAM_RANKS[F][q], ss[q]) : 0; \
        }                                                                                 \
        ++n;                                                                              \
    } while (0)
    for (int s = 0; s < nr; ++s) EMIT(1, s, 0, 0);
    for (int F = 2; F <= 4; ++F)
        for (int s1 = 0; s1 < nr; ++s1) for (int s2 = s1; s2 < nr; ++s2) EMIT(F, s1, s2, 0);
    for (int s1 = 0; s1 < nr; ++s1) for (int s2 = s1; s2 < nr; ++s2) for (int s3 = s2; s3 < nr; ++s3)
        EMIT(5, s1, s2, s3);
    for (int s1 = 0; s1 < nr; ++s1) for (int s2 = 0; s2 < nr; ++s2) for (int s3 = s1; s3 < nr; ++s3)
        EMIT(6, s1, s2, s3);
    for (int s1 = 0; s1 < nr; ++s1) for (int s2 = s1; s2 < nr; ++s2) for (int s3 = 0; s3 < nr; ++s3)
        EMIT(7, s1, s2, s3);
    for (int s1 = 0; s1 < nr; ++s1) for (int s2 = 0; s2 < nr; ++s2) for (int s3 = 0; s3 < nr; ++s3)
        EMIT(8, s1, s2, s3);
#undef EMIT
    return n;
}

/* ------------------------------------------------------------------ network */

static double act(int kind, double z, double *d1, double *d2) {
    if (kind == 0) {
        double t = tanh(z);
        *d1 = 1.0 - t * t;
        *d2 = -2.0 * t * (*d1);
        return t;
    }
    double s = 1.0 / (1.0 + exp(-z));
    *d1 = s * (1.0 + z * (1.0 - s));
    *d2 = s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s));
    return z * s;
}

/* ------------------------------------------------------------------ shared per-atom */

typedef struct {
    int nf, nr, nt;
    feature *ft;
} ctx_t;

static void ctx_init(const or_model *M, ctx_t *cx) {
    cx->nr = M->n_radial;
    cx->nt = OR_NT(M->n_radial);
    cx->nf = or_feature_table(cx->nr, NULL, NULL);
    int *fam = (int *)malloc(sizeof(int) * cx->nf), *off = (int *)malloc(sizeof(int) * 3 * cx->nf);
    or_feature_table(cx->nr, fam, off);
    cx->ft = (feature *)malloc(sizeof(feature) * cx->nf);
    for (int f = 0; f < cx->nf; ++f) {
        cx->ft[f].fam = fam[f];
        for (int q = 0; q < 3; ++q) cx->ft[f].off[q] = off[3 * f + q];
    }
    free(fam);
    free(off);
}
static void ctx_free(ctx_t *cx) { free(cx->ft); }

/* displacement d = (x_j - x_i) + shift . cell */
static void displacement(const double *pos, const double *C, int i, int j, const int *sh, double *d) {
    for (int c = 0; c < 3; ++c)
        d[c] = (pos[3 * j + c] - pos[3 * i + c]) + (sh[0] * C[c] + sh[1] * C[3 + c] + sh[2] * C[6 + c]);
}

/* radial functions R_s and dR_s/dr of an ordered species pair */
static void radial(const or_model *M, int zi, int zj, const pair_basis *pb, double *R, double *dR) {
    const int nb = M->n_basis, nr = M->n_radial;
    const double norm = 1.0 / sqrt((double)nb);
    const double *bt = M->beta + ((size_t)zi * M->n_species + zj) * nr * nb;
    for (int s = 0; s < nr; ++s) {
        double v = 0.0, dv = 0.0;
        for (int k = 0; k < nb; ++k) { v += bt[s * nb + k] * pb->B[k]; dv += bt[s * nb + k] * pb->dB[k]; }
        R[s] = v * norm;
        dR[s] = dv * norm;
    }
}

static int struct_of(int n_struct, const int *atom_ptr, int i) {
    int lo = 0, hi = n_struct - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (atom_ptr[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* Test hooks for the pins of the radial part (section "Machine Learning Interatomic
 * Potentials": basis functions combined by species-pair coefficients into R).
 * or_radial_basis: B[k] = f_c(r) Phi_k(r) and dB[k] = d/dr of it, k < n_basis.
 * or_radial_fns:   R[s] and dR[s]/dr of the ordered species pair (zi, zj), s < n_radial. */
int or_radial_basis(const or_model *M, double r, double *B, double *dB) {
    if (M->n_basis > 16) return 2;
    pair_basis pb;
    basis_eval(M, r, &pb);
    for (int k = 0; k < M->n_basis; ++k) {
        B[k] = pb.B[k];
        dB[k] = pb.dB[k];
    }
    return 0;
}

int or_radial_fns(const or_model *M, int zi, int zj, double r, double *R, double *dR) {
    if (M->n_basis > 16 || M->n_radial > OR_MAXR) return 2;
    if (zi < 0 || zj < 0 || zi >= M->n_species || zj >= M->n_species) return 3;
    pair_basis pb;
    basis_eval(M, r, &pb);
    radial(M, zi, zj, &pb, R, dR);
    return 0;
}

/* ------------------------------------------------------------------ energy + forces */

/*
 * or_energy_forces: energies E_struct[B], per-atom energies E_atom[N] (or NULL),
 * forces F[N*3], virial[B*9] (or NULL), unique-component moments psi_out[N][nr][20]
 * (or NULL) and features G_out[N][nf] (or NULL), given a CSR neighbour list
 * (row_ptr[N+1], col[P], shift[P*3], shifts relative to pos).
 */
int or_energy_forces(const or_model *M, int n_struct, const int *atom_ptr, const double *pos,
                     const int *species, const double *cell, const int64_t *row_ptr, const int *col,
                     const int *shift, double *E_struct, double *E_atom, double *F, double *virial,
                     double *psi_out, double *G_out) {
    if (M->n_radial > OR_MAXR || M->n_basis > 16) return 2;
    const int N = atom_ptr[n_struct];
    ctx_t cx;
    ctx_init(M, &cx);
    const int nr = cx.nr, nt = cx.nt, nf = cx.nf, H = M->n_hidden;
    const int64_t P = row_ptr[N];
    double *gpair = (double *)calloc((size_t)3 * (P ? P : 1), sizeof(double));
    double *Ea = (double *)calloc(N ? N : 1, sizeof(double));
    int err = 0;

#pragma omp parallel
    {
        double *T = (double *)malloc(sizeof(double) * nt), *Tb = (double *)malloc(sizeof(double) * nt);
        double *G = (double *)malloc(sizeof(double) * nf), *Gb = (double *)malloc(sizeof(double) * nf);
        double *z1 = (double *)malloc(sizeof(double) * H), *a1 = (double *)malloc(sizeof(double) * H);
        double *d1 = (double *)malloc(sizeof(double) * H), *z2 = (double *)malloc(sizeof(double) * H);
        double *a2 = (double *)malloc(sizeof(double) * H), *d2 = (double *)malloc(sizeof(double) * H);
        double *ab = (double *)malloc(sizeof(double) * H), *zb = (double *)malloc(sizeof(double) * H);
        double Y[4][27], dY[4][27][3], R[OR_MAXR], dR[OR_MAXR];
        pair_basis pb;
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < N; ++i) {
            const int b = struct_of(n_struct, atom_ptr, i);
            const double *C = cell + 9 * b;
            const int zi = species[i];
            memset(T, 0, sizeof(double) * nt);
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double d[3];
                const int j = col[p];
                displacement(pos, C, i, j, shift + 3 * p, d);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                basis_eval(M, r, &pb);
                radial(M, zi, species[j], &pb, R, dR);
                double u[3] = {d[0] / r, d[1] / r, d[2] / r};
                monomials(u, r, Y, dY);
                for (int s = 0; s < nr; ++s)
                    for (int L = 0; L < 4; ++L) {
                        double *t = T + toff(nr, L, s);
                        for (int q = 0; q < TSIZE[L]; ++q) t[q] += R[s] * Y[L][q];
                    }
            }
            for (int f = 0; f < nf; ++f)
                G[f] = fam_val(cx.ft[f].fam, T + cx.ft[f].off[0], T + cx.ft[f].off[1], T + cx.ft[f].off[2]);
            /* network forward */
            for (int h = 0; h < H; ++h) {
                double z = M->b1[h];
                for (int f = 0; f < nf; ++f) z += G[f] * M->W1[(size_t)f * H + h];
                double dd, d2d;
                z1[h] = z;
                a1[h] = act(M->activation, z, &dd, &d2d);
                d1[h] = dd;
            }
            double nn = M->b3[0];
            for (int h = 0; h < H; ++h) {
                double z = M->b2[h];
                for (int g = 0; g < H; ++g) z += a1[g] * M->W2[(size_t)g * H + h];
                double dd, d2d;
                z2[h] = z;
                a2[h] = act(M->activation, z, &dd, &d2d);
                d2[h] = dd;
                nn += M->w3[h] * a2[h];
            }
            Ea[i] = M->sigma[zi] * nn + M->mu[zi];
            /* network backward: dE/dG */
            for (int h = 0; h < H; ++h) zb[h] = M->sigma[zi] * M->w3[h] * d2[h];
            for (int g = 0; g < H; ++g) {
                double s = 0.0;
                for (int h = 0; h < H; ++h) s += M->W2[(size_t)g * H + h] * zb[h];
                ab[g] = s * d1[g];
            }
            for (int f = 0; f < nf; ++f) {
                double s = 0.0;
                for (int h = 0; h < H; ++h) s += M->W1[(size_t)f * H + h] * ab[h];
                Gb[f] = s;
            }
            /* contraction backward: dE/dT */
            memset(Tb, 0, sizeof(double) * nt);
            for (int f = 0; f < nf; ++f) {
                const feature *ft = &cx.ft[f];
                const int ar = FAM_ARITY[ft->fam];
                fam_grad(ft->fam, T + ft->off[0], T + ft->off[1], T + ft->off[2], Gb[f], Tb + ft->off[0],
                         ar > 1 ? Tb + ft->off[1] : NULL, ar > 2 ? Tb + ft->off[2] : NULL);
            }
            /* per-pair gradients g_ij = dE/dd_ij */
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double d[3];
                const int j = col[p];
                displacement(pos, C, i, j, shift + 3 * p, d);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                basis_eval(M, r, &pb);
                radial(M, zi, species[j], &pb, R, dR);
                double u[3] = {d[0] / r, d[1] / r, d[2] / r};
                monomials(u, r, Y, dY);
                double g[3] = {0, 0, 0};
                for (int s = 0; s < nr; ++s)
                    for (int L = 0; L < 4; ++L) {
                        const double *tb = Tb + toff(nr, L, s);
                        for (int q = 0; q < TSIZE[L]; ++q)
                            for (int c = 0; c < 3; ++c)
                                g[c] += tb[q] * (dR[s] * u[c] * Y[L][q] + R[s] * dY[L][q][c]);
                    }
                for (int c = 0; c < 3; ++c) gpair[3 * p + c] = g[c];
            }
            if (psi_out) {
                double *po = psi_out + (size_t)i * nr * 20;
                static const int I2[6] = {0, 1, 2, 4, 5, 8};
                static const int I3[10] = {0, 1, 2, 4, 5, 8, 13, 14, 17, 26};
                for (int s = 0; s < nr; ++s) {
                    po[20 * s] = T[toff(nr, 0, s)];
                    for (int a = 0; a < 3; ++a) po[20 * s + 1 + a] = T[toff(nr, 1, s) + a];
                    for (int a = 0; a < 6; ++a) po[20 * s + 4 + a] = T[toff(nr, 2, s) + I2[a]];
                    for (int a = 0; a < 10; ++a) po[20 * s + 10 + a] = T[toff(nr, 3, s) + I3[a]];
                }
            }
            if (G_out) memcpy(G_out + (size_t)i * nf, G, sizeof(double) * nf);
        }
        free(T); free(Tb); free(G); free(Gb); free(z1); free(a1); free(d1); free(z2); free(a2); free(d2);
        free(ab); free(zb);
    }
    /* assemble forces F_i = sum_j g_ij - sum_{(j,i)} g_ji, energies and virials */
    memset(F, 0, sizeof(double) * 3 * N);
    for (int b = 0; b < n_struct; ++b) {
        double e = 0.0;
        for (int i = atom_ptr[b]; i < atom_ptr[b + 1]; ++i) e += Ea[i];
        E_struct[b] = e;
        if (virial) memset(virial + 9 * b, 0, sizeof(double) * 9);
    }
    for (int i = 0; i < N; ++i) {
        const int b = struct_of(n_struct, atom_ptr, i);
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const int j = col[p];
            for (int c = 0; c < 3; ++c) {
                F[3 * i + c] += gpair[3 * p + c];
                F[3 * j + c] -= gpair[3 * p + c];
            }
            if (virial) {
                double d[3];
                displacement(pos, cell + 9 * b, i, j, shift + 3 * p, d);
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) virial[9 * b + 3 * a + c] -= d[a] * gpair[3 * p + c];
            }
        }
    }
    if (E_atom) memcpy(E_atom, Ea, sizeof(double) * N);
    free(gpair);
    free(Ea);
    ctx_free(&cx);
    return err;
}

/* ------------------------------------------------------------------ descriptors */

/* Moments (unique components, [nr][20]) and features of the atoms listed in rows[],
 * from their CSR rows (other rows are ignored).  Same arithmetic as or_energy_forces. */
int or_descriptors(const or_model *M, int n_struct, const int *atom_ptr, const double *pos, const int *species,
                   const double *cell, const int64_t *row_ptr, const int *col, const int *shift, int n_rows,
                   const int *rows, double *psi_out, double *G_out) {
    if (M->n_radial > OR_MAXR || M->n_basis > 16) return 2;
    ctx_t cx;
    ctx_init(M, &cx);
    const int nr = cx.nr, nt = cx.nt, nf = cx.nf;
#pragma omp parallel
    {
        double *T = (double *)malloc(sizeof(double) * nt);
        double Y[4][27], dY[4][27][3], R[OR_MAXR], dR[OR_MAXR];
        pair_basis pb;
        static const int I2[6] = {0, 1, 2, 4, 5, 8};
        static const int I3[10] = {0, 1, 2, 4, 5, 8, 13, 14, 17, 26};
#pragma omp for schedule(dynamic, 4)
        for (int q = 0; q < n_rows; ++q) {
            const int i = rows[q];
            const double *C = cell + 9 * struct_of(n_struct, atom_ptr, i);
            memset(T, 0, sizeof(double) * nt);
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double d[3];
                const int j = col[p];
                displacement(pos, C, i, j, shift + 3 * p, d);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                basis_eval(M, r, &pb);
                radial(M, species[i], species[j], &pb, R, dR);
                double u[3] = {d[0] / r, d[1] / r, d[2] / r};
                monomials(u, r, Y, dY);
                for (int s = 0; s < nr; ++s)
                    for (int L = 0; L < 4; ++L) {
                        double *t = T + toff(nr, L, s);
                        for (int c = 0; c < TSIZE[L]; ++c) t[c] += R[s] * Y[L][c];
                    }
            }
            double *po = psi_out + (size_t)q * nr * 20;
            for (int s = 0; s < nr; ++s) {
                po[20 * s] = T[toff(nr, 0, s)];
                for (int a = 0; a < 3; ++a) po[20 * s + 1 + a] = T[toff(nr, 1, s) + a];
                for (int a = 0; a < 6; ++a) po[20 * s + 4 + a] = T[toff(nr, 2, s) + I2[a]];
                for (int a = 0; a < 10; ++a) po[20 * s + 10 + a] = T[toff(nr, 3, s) + I3[a]];
            }
            for (int f = 0; f < nf; ++f)
                G_out[(size_t)q * nf + f] =
                    fam_val(cx.ft[f].fam, T + cx.ft[f].off[0], T + cx.ft[f].off[1], T + cx.ft[f].off[2]);
        }
        free(T);
    }
    ctx_free(&cx);
    return 0;
}

/* ------------------------------------------------------------------ loss */

/* Force-matching loss and its gradients with respect to E_b and F_i. */
double or_loss(int n_struct, const int *atom_ptr, const double *E, const double *E_ref, const double *F,
               const double *F_ref, double wE, double wF, double *gE, double *gF) {
    const int N = atom_ptr[n_struct];
    double le = 0.0, lf = 0.0;
    for (int b = 0; b < n_struct; ++b) {
        double nb = atom_ptr[b + 1] - atom_ptr[b];
        double e = (E[b] - E_ref[b]) / nb;
        le += e * e;
        if (gE) gE[b] = 2.0 * wE / n_struct * e / nb;
    }
    for (int q = 0; q < 3 * N; ++q) {
        double e = F[q] - F_ref[q];
        lf += e * e;
        if (gF) gF[q] = 2.0 * wF / (3.0 * N) * e;
    }
    return wE / n_struct * le + wF / (3.0 * N) * lf;
}

/* ------------------------------------------------------------------ parameter gradient */

/*
 * or_param_grad: gradient of J(theta) = sum_b gE[b] E_b + sum_i gF[i] . F_i with respect
 * to every parameter (the chain rule of a loss through E and F).  Since
 * F = -dE/dr, sum_i v_i . F_i = -(d/dt) E(r + t v) with v = gF, so J is evaluated per
 * atom as gE_b E_i - dE_i/dt: a forward pass carrying the primal and the tangent along
 * v, followed by a reverse pass through both.  Outputs are overwritten.
 */
int or_param_grad(const or_model *M, int n_struct, const int *atom_ptr, const double *pos,
                  const int *species, const double *cell, const int64_t *row_ptr, const int *col,
                  const int *shift, const double *gE, const double *gF, const or_grad *out) {
    if (M->n_radial > OR_MAXR || M->n_basis > 16) return 2;
    const int N = atom_ptr[n_struct];
    ctx_t cx;
    ctx_init(M, &cx);
    const int nr = cx.nr, nt = cx.nt, nf = cx.nf, H = M->n_hidden, S = M->n_species, nb = M->n_basis;
    const size_t nbeta = (size_t)S * S * nr * nb, nW1 = (size_t)nf * H, nW2 = (size_t)H * H;
    const size_t ntot = nbeta + nW1 + H + nW2 + H + H + 1 + S + S;
    double *acc_all = NULL;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    acc_all = (double *)calloc((size_t)nthreads * ntot, sizeof(double));
    const double norm = 1.0 / sqrt((double)nb);

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *acc = acc_all + (size_t)tid * ntot;
        double *gbeta = acc, *gW1 = gbeta + nbeta, *gb1 = gW1 + nW1, *gW2 = gb1 + H, *gb2 = gW2 + nW2;
        double *gw3 = gb2 + H, *gb3 = gw3 + H, *gsig = gb3 + 1, *gmu = gsig + S;
        double *T = (double *)malloc(sizeof(double) * nt), *Td = (double *)malloc(sizeof(double) * nt);
        double *Tb = (double *)malloc(sizeof(double) * nt), *Tdb = (double *)malloc(sizeof(double) * nt);
        double *G = (double *)malloc(sizeof(double) * nf), *Gd = (double *)malloc(sizeof(double) * nf);
        double *Gb = (double *)malloc(sizeof(double) * nf), *Gdb = (double *)malloc(sizeof(double) * nf);
        double *buf = (double *)malloc(sizeof(double) * H * 16);
        double *z1 = buf, *z1d = buf + H, *a1 = buf + 2 * H, *a1d = buf + 3 * H, *p1 = buf + 4 * H,
               *q1 = buf + 5 * H, *z2 = buf + 6 * H, *z2d = buf + 7 * H, *a2 = buf + 8 * H,
               *a2d = buf + 9 * H, *p2 = buf + 10 * H, *q2 = buf + 11 * H, *z2b = buf + 12 * H,
               *z2db = buf + 13 * H, *z1b = buf + 14 * H, *z1db = buf + 15 * H;
        double Y[4][27], dY[4][27][3], R[OR_MAXR], dR[OR_MAXR];
        pair_basis pb;
#pragma omp for schedule(dynamic, 16)
        for (int i = 0; i < N; ++i) {
            const int b = struct_of(n_struct, atom_ptr, i);
            const double *C = cell + 9 * b;
            const int zi = species[i];
            const double c_i = gE[b];
            memset(T, 0, sizeof(double) * nt);
            memset(Td, 0, sizeof(double) * nt);
            /* primal and tangent moments */
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double d[3], dd[3];
                const int j = col[p];
                displacement(pos, C, i, j, shift + 3 * p, d);
                for (int c = 0; c < 3; ++c) dd[c] = gF[3 * j + c] - gF[3 * i + c];
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                basis_eval(M, r, &pb);
                radial(M, zi, species[j], &pb, R, dR);
                double u[3] = {d[0] / r, d[1] / r, d[2] / r};
                monomials(u, r, Y, dY);
                for (int s = 0; s < nr; ++s)
                    for (int L = 0; L < 4; ++L) {
                        double *t = T + toff(nr, L, s), *td = Td + toff(nr, L, s);
                        for (int q = 0; q < TSIZE[L]; ++q) {
                            t[q] += R[s] * Y[L][q];
                            double dir = 0.0;
                            for (int c = 0; c < 3; ++c) dir += dd[c] * (dR[s] * u[c] * Y[L][q] + R[s] * dY[L][q][c]);
                            td[q] += dir;
                        }
                    }
            }
            /* features and their tangents (multilinearity) */
            for (int f = 0; f < nf; ++f) {
                const feature *ft = &cx.ft[f];
                const double *A = T + ft->off[0], *B = T + ft->off[1], *Cc = T + ft->off[2];
                const double *Ad = Td + ft->off[0], *Bd = Td + ft->off[1], *Cd = Td + ft->off[2];
                const int ar = FAM_ARITY[ft->fam];
                G[f] = fam_val(ft->fam, A, B, Cc);
                double gd = fam_val(ft->fam, Ad, B, Cc);
                if (ar > 1) gd += fam_val(ft->fam, A, Bd, Cc);
                if (ar > 2) gd += fam_val(ft->fam, A, B, Cd);
                Gd[f] = gd;
            }
            /* network: primal and tangent */
            for (int h = 0; h < H; ++h) {
                double z = M->b1[h], zd = 0.0;
                for (int f = 0; f < nf; ++f) { z += G[f] * M->W1[(size_t)f * H + h]; zd += Gd[f] * M->W1[(size_t)f * H + h]; }
                z1[h] = z; z1d[h] = zd;
                a1[h] = act(M->activation, z, &p1[h], &q1[h]);
                a1d[h] = p1[h] * zd;
            }
            double nn = M->b3[0], nnd = 0.0;
            for (int h = 0; h < H; ++h) {
                double z = M->b2[h], zd = 0.0;
                for (int g = 0; g < H; ++g) { z += a1[g] * M->W2[(size_t)g * H + h]; zd += a1d[g] * M->W2[(size_t)g * H + h]; }
                z2[h] = z; z2d[h] = zd;
                a2[h] = act(M->activation, z, &p2[h], &q2[h]);
                a2d[h] = p2[h] * zd;
                nn += M->w3[h] * a2[h];
                nnd += M->w3[h] * a2d[h];
            }
            /* reverse pass of j_i = c_i E_i - dE_i/dt,  E_i = sigma nn + mu */
            const double sg = M->sigma[zi];
            gsig[zi] += c_i * nn - nnd;
            gmu[zi] += c_i;
            const double nnb = c_i * sg, nndb = -sg;
            gb3[0] += nnb;
            for (int h = 0; h < H; ++h) {
                gw3[h] += nnb * a2[h] + nndb * a2d[h];
                const double a2b = nnb * M->w3[h], a2db = nndb * M->w3[h];
                z2db[h] = p2[h] * a2db;
                z2b[h] = q2[h] * z2d[h] * a2db + p2[h] * a2b;
                gb2[h] += z2b[h];
            }
            for (int g = 0; g < H; ++g) {
                double a1b = 0.0, a1db = 0.0;
                for (int h = 0; h < H; ++h) {
                    const double w = M->W2[(size_t)g * H + h];
                    gW2[(size_t)g * H + h] += a1[g] * z2b[h] + a1d[g] * z2db[h];
                    a1b += w * z2b[h];
                    a1db += w * z2db[h];
                }
                z1db[g] = p1[g] * a1db;
                z1b[g] = q1[g] * z1d[g] * a1db + p1[g] * a1b;
                gb1[g] += z1b[g];
            }
            for (int f = 0; f < nf; ++f) {
                double gb = 0.0, gdb = 0.0;
                for (int h = 0; h < H; ++h) {
                    const double w = M->W1[(size_t)f * H + h];
                    gW1[(size_t)f * H + h] += G[f] * z1b[h] + Gd[f] * z1db[h];
                    gb += w * z1b[h];
                    gdb += w * z1db[h];
                }
                Gb[f] = gb;
                Gdb[f] = gdb;
            }
            /* contraction adjoints: primal Tb and tangent Tdb */
            memset(Tb, 0, sizeof(double) * nt);
            memset(Tdb, 0, sizeof(double) * nt);
            for (int f = 0; f < nf; ++f) {
                const feature *ft = &cx.ft[f];
                const int fam = ft->fam, ar = FAM_ARITY[fam];
                const int o0 = ft->off[0], o1 = ft->off[1], o2 = ft->off[2];
                /* value term: Tb += Gb * grad f(T) */
                fam_grad(fam, T + o0, T + o1, T + o2, Gb[f], Tb + o0, ar > 1 ? Tb + o1 : NULL,
                         ar > 2 ? Tb + o2 : NULL);
                /* tangent term  Gd = sum_k f(.., Td_k, ..): each summand feeds Tdb at its
                 * tangent slot and Tb at the other slots */
                fam_grad(fam, Td + o0, T + o1, T + o2, Gdb[f], Tdb + o0, ar > 1 ? Tb + o1 : NULL,
                         ar > 2 ? Tb + o2 : NULL);
                if (ar > 1)
                    fam_grad(fam, T + o0, Td + o1, T + o2, Gdb[f], Tb + o0, Tdb + o1, ar > 2 ? Tb + o2 : NULL);
                if (ar > 2)
                    fam_grad(fam, T + o0, T + o1, Td + o2, Gdb[f], Tb + o0, Tb + o1, Tdb + o2);
            }
            /* species-pair coefficients */
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                double d[3], dd[3];
                const int j = col[p];
                displacement(pos, C, i, j, shift + 3 * p, d);
                for (int c = 0; c < 3; ++c) dd[c] = gF[3 * j + c] - gF[3 * i + c];
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                basis_eval(M, r, &pb);
                double u[3] = {d[0] / r, d[1] / r, d[2] / r};
                monomials(u, r, Y, dY);
                double *gb_pair = gbeta + ((size_t)zi * S + species[j]) * nr * nb;
                for (int s = 0; s < nr; ++s)
                    for (int k = 0; k < nb; ++k) {
                        double v = 0.0;
                        for (int L = 0; L < 4; ++L) {
                            const double *tb = Tb + toff(nr, L, s), *tdb = Tdb + toff(nr, L, s);
                            for (int q = 0; q < TSIZE[L]; ++q) {
                                double dir = 0.0;
                                for (int c = 0; c < 3; ++c)
                                    dir += dd[c] * (pb.dB[k] * u[c] * Y[L][q] + pb.B[k] * dY[L][q][c]);
                                v += tb[q] * pb.B[k] * Y[L][q] + tdb[q] * dir;
                            }
                        }
                        gb_pair[s * nb + k] += v * norm;
                    }
            }
        }
        free(T); free(Td); free(Tb); free(Tdb); free(G); free(Gd); free(Gb); free(Gdb); free(buf);
    }
    /* reduce the per-thread accumulators in thread order */
    double *dst[9] = {out->beta, out->W1, out->b1, out->W2, out->b2, out->w3, out->b3, out->sigma, out->mu};
    size_t len[9] = {nbeta, nW1, (size_t)H, nW2, (size_t)H, (size_t)H, 1, (size_t)S, (size_t)S};
    size_t off = 0;
    for (int q = 0; q < 9; ++q) {
        for (size_t e = 0; e < len[q]; ++e) {
            double s = 0.0;
            for (int t = 0; t < nthreads; ++t) s += acc_all[(size_t)t * ntot + off + e];
            dst[q][e] = s;
        }
        off += len[q];
    }
    free(acc_all);
    ctx_free(&cx);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel loops (timing on a given number of host cores). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
