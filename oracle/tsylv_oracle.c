/*
 * Plain CPU FP64 oracle for the (quasi-)triangular tensor Sylvester equation.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the solver library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no code with the CUDA path.
 *
 * Problem (Chen & Kressner, "Recursive blocked algorithms for linear systems
 * with Kronecker product structure"):
 *   Laplace-like form, Sec. 2, Eq. (2.2):  sum_mu X x_mu A_mu = B
 *   d-term generalized form (Conclusions, the K-term equation with K = d and
 *   mode family {A_mu, C_mu}):  sum_mu X x_mu A_mu x_{eta != mu} C_eta = B
 * with A_mu upper quasi-triangular (1x1 and 2x2 diagonal blocks, Sec. 2 after
 * Alg. 1) and C_mu upper triangular.  C == NULL means C_mu = I (Laplace form).
 *
 * Layout: a d-way tensor is stored column-major, mode 1 fastest (the index
 * map of Eq. (2.1)); an n x n matrix M is column-major, M(i,j) = M[i + n*j].
 * The mode-mu product Y = X x_mu M is defined by Y_(mu) = M X_(mu) (Sec. 2).
 *
 * Two independent solution routes:
 *  O-A  orc_backsub: element back-substitution over the coupled diagonal
 *       groups (products of the 1x1 / 2x2 diagonal blocks of every mode),
 *       visited in decreasing lexicographic order; the right-hand side of a
 *       group subtracts every already-solved unknown times the operator entry
 *       computed from its definition; the group system is solved by Gaussian
 *       elimination with partial pivoting.  This is the base case of Alg. 2
 *       (Sec. 2.1: the small block-triangular system solved by
 *       back-substitution), applied to a whole tensor.
 *  O-B  orc_recursive: Alg. 2 (Sec. 2.1) -- split the largest mode at
 *       k = floor(n_mu/2), k+1 if that cuts a 2x2 block; solve the trailing
 *       part; update the leading right-hand side (Eq. (2.3a)); solve the
 *       leading part.  The generalized update follows the term pattern of
 *       Sec. 3.1 (Case 1 / Case 2 right-hand sides) for the d-term form and is
 *       evaluated term by term.  The leaf (largest extent <= nmin) is solved by
 *       O-A on the sub-tensor.
 *
 * Return codes: 0 ok, -1 bad arguments / structure, 1 singular group pivot.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_MAXD 8

/* ---------------------------------------------------------------- helpers */

static int64_t prod_range(const int64_t* n, int lo, int hi) {
    int64_t p = 1;
    for (int i = lo; i < hi; i++) p *= n[i];
    return p;
}

/* Operator coefficient: mode eta of term mu is A_eta if eta == mu, else C_eta
 * (identity when C is NULL).  Entry (i, j), 0-based, of an n x n matrix. */
static double coef(const double* const* A, const double* const* C, int64_t ld,
                   int term, int eta, int64_t i, int64_t j) {
    if (term == eta) return A[eta][i + ld * j];
    if (C == NULL) return i == j ? 1.0 : 0.0;
    return C[eta][i + ld * j];
}

/* Structure checks (Sec. 2: upper quasi-triangular; Sec. 3.1: C upper
 * triangular).  Only A(i+1,i) may be nonzero below the diagonal, never two
 * in a row. */
int orc_check_structure(int d, const int64_t* n, const double* const* A) {
    if (d < 1 || d > ORC_MAXD) return -1;
    for (int mu = 0; mu < d; mu++) {
        if (n[mu] < 1) return -1;
        int64_t m = n[mu];
        for (int64_t i = 0; i + 2 < m; i++)
            if (A[mu][(i + 1) + m * i] != 0.0 && A[mu][(i + 2) + m * (i + 1)] != 0.0) return -1;
    }
    return 0;
}

/* Group map of mode mu: gstart[i] = first index of the diagonal block that
 * contains i, glen[i] = its size (1 or 2). */
static void group_map(const double* Amu, int64_t m, int64_t* gstart, int* glen) {
    int64_t i = 0;
    while (i < m) {
        if (i + 1 < m && Amu[(i + 1) + m * i] != 0.0) {
            gstart[i] = i; gstart[i + 1] = i; glen[i] = 2; glen[i + 1] = 2; i += 2;
        } else {
            gstart[i] = i; glen[i] = 1; i += 1;
        }
    }
}

/* Dense Gaussian elimination with partial pivoting, in place: M is s x s
 * (row-major, M[r*s+c]), rhs length s. Returns 1 if a pivot is exactly 0. */
static int gepp(int s, double* M, double* rhs) {
    for (int c = 0; c < s; c++) {
        int p = c; double best = fabs(M[c * s + c]);
        for (int r = c + 1; r < s; r++) if (fabs(M[r * s + c]) > best) { best = fabs(M[r * s + c]); p = r; }
        if (best == 0.0) return 1;
        if (p != c) {
            for (int k = 0; k < s; k++) { double t = M[c * s + k]; M[c * s + k] = M[p * s + k]; M[p * s + k] = t; }
            double t = rhs[c]; rhs[c] = rhs[p]; rhs[p] = t;
        }
        for (int r = c + 1; r < s; r++) {
            double f = M[r * s + c] / M[c * s + c];
            if (f == 0.0) continue;
            for (int k = c; k < s; k++) M[r * s + k] -= f * M[c * s + k];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = s - 1; c >= 0; c--) {
        double v = rhs[c];
        for (int k = c + 1; k < s; k++) v -= M[c * s + k] * rhs[k];
        rhs[c] = v / M[c * s + c];
    }
    return 0;
}

/* ------------------------------------------------------ operator (Eq. 2.2) */

/* Y = X x_mu M restricted: output rows [r0, r0+nr) of mode mu come from input
 * rows [c0, c0+nc) of mode mu through M(r, c) = M[(mrow0 + r) + ldm*(mcol0 + c)].
 * X has extents nx (mode mu extent nc), Y has extents ny = nx with mode mu -> nr.
 * This is the definition Y_(mu) = M X_(mu) on a sub-block of M. */
static void mode_product_block(int d, const int64_t* nx, int mu, const double* M, int64_t ldm,
                               int64_t mrow0, int64_t mcol0, int64_t nr, int transpose,
                               const double* X, double* Y) {
    int64_t L = prod_range(nx, 0, mu), nc = nx[mu], R = prod_range(nx, mu + 1, d);
    for (int64_t r = 0; r < R; r++)
        for (int64_t ip = 0; ip < nr; ip++)
            for (int64_t l = 0; l < L; l++) {
                double s = 0.0;
                for (int64_t i = 0; i < nc; i++) {
                    double mv = transpose ? M[(mcol0 + i) + ldm * (mrow0 + ip)]
                                          : M[(mrow0 + ip) + ldm * (mcol0 + i)];
                    if (mv != 0.0) s += mv * X[l + L * (i + nc * r)];
                }
                Y[l + L * (ip + nr * r)] = s;
            }
}

/* Y = A(X) (transpose = 0) or A^T(X) (transpose = 1), the full operator of the
 * Laplace form (C == NULL, Eq. (2.2)) or of the d-term generalized form.
 * Term by term: T_mu = X x_1 M_{mu,1} ... x_d M_{mu,d}. */
int orc_apply(int d, const int64_t* n, const double* const* A, const double* const* C,
              const double* X, double* Y, int transpose) {
    if (d < 1 || d > ORC_MAXD) return -1;
    int64_t N = prod_range(n, 0, d);
    double* t0 = (double*)malloc(sizeof(double) * (size_t)N);
    double* t1 = (double*)malloc(sizeof(double) * (size_t)N);
    if (!t0 || !t1) { free(t0); free(t1); return -1; }
    memset(Y, 0, sizeof(double) * (size_t)N);
    for (int term = 0; term < d; term++) {
        memcpy(t0, X, sizeof(double) * (size_t)N);
        for (int eta = 0; eta < d; eta++) {
            const double* M;
            if (eta == term) M = A[eta];
            else if (C == NULL) continue;           /* identity factor */
            else M = C[eta];
            mode_product_block(d, n, eta, M, n[eta], 0, 0, n[eta], transpose, t0, t1);
            double* t = t0; t0 = t1; t1 = t;
        }
        for (int64_t q = 0; q < N; q++) Y[q] += t0[q];
    }
    free(t0); free(t1);
    return 0;
}

/* Operator entry between positions u and v (full-tensor indices), from the
 * Kronecker representation Eq. (1.4) (Laplace) or its d-term analogue:
 *   op(u, v) = sum_mu prod_eta M_{mu,eta}(u_eta, v_eta). */
static double op_entry(int d, const int64_t* n, const double* const* A, const double* const* C,
                       const int64_t* u, const int64_t* v) {
    double s = 0.0;
    for (int term = 0; term < d; term++) {
        double p = 1.0;
        for (int eta = 0; eta < d && p != 0.0; eta++) p *= coef(A, C, n[eta], term, eta, u[eta], v[eta]);
        s += p;
    }
    return s;
}

/* ------------------------------------------------- O-A: back-substitution */

typedef struct {
    int d; const int64_t* n; int64_t st[ORC_MAXD];
    const double* const* A; const double* const* C;
    int64_t* gstart[ORC_MAXD]; int* glen[ORC_MAXD];
} orc_ctx;

static int ctx_init(orc_ctx* c, int d, const int64_t* n, const double* const* A, const double* const* C) {
    c->d = d; c->n = n; c->A = A; c->C = C;
    int64_t s = 1;
    for (int mu = 0; mu < d; mu++) { c->st[mu] = s; s *= n[mu]; c->gstart[mu] = NULL; c->glen[mu] = NULL; }
    for (int mu = 0; mu < d; mu++) {
        c->gstart[mu] = (int64_t*)malloc(sizeof(int64_t) * (size_t)n[mu]);
        c->glen[mu] = (int*)malloc(sizeof(int) * (size_t)n[mu]);
        if (!c->gstart[mu] || !c->glen[mu]) return -1;
        group_map(A[mu], n[mu], c->gstart[mu], c->glen[mu]);
    }
    return 0;
}
static void ctx_free(orc_ctx* c) {
    for (int mu = 0; mu < c->d; mu++) { free(c->gstart[mu]); free(c->glen[mu]); }
}

static int64_t lin(const orc_ctx* c, const int64_t* u) {
    int64_t q = 0;
    for (int mu = 0; mu < c->d; mu++) q += u[mu] * c->st[mu];
    return q;
}

/* Solve the sub-problem on the box [off, off+ext) of X in place (X holds the
 * right-hand side of that box on entry, already updated for everything
 * outside the box).  transpose = 1 solves A^T (forward substitution: groups in
 * increasing order, entries op(v, u)). */
static int backsub_box(const orc_ctx* c, double* X, const int64_t* off, const int64_t* ext, int transpose) {
    int d = c->d;
    int64_t g[ORC_MAXD];                  /* current group start per mode */
    /* enumerate groups of each mode inside the box */
    int64_t* gl[ORC_MAXD]; int ng[ORC_MAXD];
    for (int mu = 0; mu < d; mu++) {
        gl[mu] = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ext[mu] + 1));
        ng[mu] = 0;
        for (int64_t i = off[mu]; i < off[mu] + ext[mu];) {
            if (c->gstart[mu][i] != i || i + c->glen[mu][i] > off[mu] + ext[mu]) {
                for (int q = 0; q <= mu; q++) free(gl[q]);
                return -1;                /* box cuts a 2x2 block */
            }
            gl[mu][ng[mu]++] = i; i += c->glen[mu][i];
        }
    }
    int gi[ORC_MAXD];
    for (int mu = 0; mu < d; mu++) gi[mu] = transpose ? 0 : ng[mu] - 1;
    int status = 0;
    double* sys = (double*)malloc(sizeof(double) * 65536);
    double* rhs = (double*)malloc(sizeof(double) * 256);
    int64_t (*pos)[ORC_MAXD] = malloc(sizeof(int64_t[ORC_MAXD]) * 256);
    for (;;) {
        /* positions of this group */
        int s = 1, sz[ORC_MAXD];
        for (int mu = 0; mu < d; mu++) { g[mu] = gl[mu][gi[mu]]; sz[mu] = c->glen[mu][g[mu]]; s *= sz[mu]; }
        for (int p = 0; p < s; p++) {
            int r = p;
            for (int mu = 0; mu < d; mu++) { pos[p][mu] = g[mu] + r % sz[mu]; r /= sz[mu]; }
        }
        /* right-hand side: subtract every solved unknown of the box.
         * Not transposed: solved = box positions in groups after this one
         * that the operator couples, i.e. v >= group start in every mode and
         * v outside the group.  Transposed: v <= group end in every mode. */
        for (int p = 0; p < s; p++) {
            const int64_t* u = pos[p];
            double acc = X[lin(c, u)];
            int64_t v[ORC_MAXD], lo[ORC_MAXD], hi[ORC_MAXD];
            for (int mu = 0; mu < d; mu++) {
                if (!transpose) { lo[mu] = g[mu]; hi[mu] = off[mu] + ext[mu]; }
                else { lo[mu] = off[mu]; hi[mu] = g[mu] + sz[mu]; }
                v[mu] = lo[mu];
            }
            if (c->C == NULL) {
                /* Laplace form: the Kronecker sum Eq. (1.4) couples u only with
                 * positions on one of its mode lines, v = u except in mode mu */
                for (int mu = 0; mu < d; mu++) {
                    for (int q = 0; q < d; q++) v[q] = u[q];
                    for (int64_t k = lo[mu]; k < hi[mu]; k++) {
                        if (k >= g[mu] && k < g[mu] + sz[mu]) continue;   /* inside the group */
                        v[mu] = k;
                        double e = transpose ? op_entry(d, c->n, c->A, c->C, v, u)
                                             : op_entry(d, c->n, c->A, c->C, u, v);
                        if (e != 0.0) acc -= e * X[lin(c, v)];
                    }
                }
                rhs[p] = acc;
                continue;
            }
            for (;;) {
                int in_group = 1;
                for (int mu = 0; mu < d; mu++) if (v[mu] < g[mu] || v[mu] >= g[mu] + sz[mu]) { in_group = 0; break; }
                if (!in_group) {
                    /* Laplace: only positions on a mode line of u couple */
                    int diff = 0;
                    if (c->C == NULL) for (int mu = 0; mu < d; mu++) diff += (v[mu] != u[mu]);
                    if (c->C != NULL || diff == 1) {
                        double e = transpose ? op_entry(d, c->n, c->A, c->C, v, u)
                                             : op_entry(d, c->n, c->A, c->C, u, v);
                        if (e != 0.0) acc -= e * X[lin(c, v)];
                    }
                }
                int mu = 0;
                while (mu < d) { if (++v[mu] < hi[mu]) break; v[mu] = lo[mu]; mu++; }
                if (mu == d) break;
            }
            rhs[p] = acc;
        }
        for (int p = 0; p < s; p++)
            for (int q = 0; q < s; q++)
                sys[p * s + q] = transpose ? op_entry(d, c->n, c->A, c->C, pos[q], pos[p])
                                           : op_entry(d, c->n, c->A, c->C, pos[p], pos[q]);
        if (gepp(s, sys, rhs)) { status = 1; break; }
        for (int p = 0; p < s; p++) X[lin(c, pos[p])] = rhs[p];
        /* next group: decreasing (increasing if transposed) lexicographic
         * order of (g_d, ..., g_1), mode 1 innermost */
        int mu = 0;
        if (!transpose) {
            while (mu < d) { if (--gi[mu] >= 0) break; gi[mu] = ng[mu] - 1; mu++; }
        } else {
            while (mu < d) { if (++gi[mu] < ng[mu]) break; gi[mu] = 0; mu++; }
        }
        if (mu == d) break;
    }
    free(sys); free(rhs); free(pos);
    for (int mu = 0; mu < d; mu++) free(gl[mu]);
    return status;
}

/* O-A on the whole tensor.  X: right-hand side on entry, solution on exit. */
int orc_backsub(int d, const int64_t* n, const double* const* A, const double* const* C,
                double* X, int transpose) {
    if (orc_check_structure(d, n, A)) return -1;
    orc_ctx c;
    if (ctx_init(&c, d, n, A, C)) { ctx_free(&c); return -1; }
    int64_t off[ORC_MAXD] = {0};
    int r = backsub_box(&c, X, off, n, transpose);
    ctx_free(&c);
    return r;
}

/* ----------------------------------------------------- O-B: Alg. 2 recursion */

typedef struct { orc_ctx c; double* X; int64_t nmin; } rec_ctx;

/* Copy the box [off, off+ext) of the full tensor X into a packed buffer (and back). */
static void box_io(const orc_ctx* c, double* X, const int64_t* off, const int64_t* ext, double* buf, int to_buf) {
    int d = c->d; int64_t v[ORC_MAXD]; int64_t q = 0;
    for (int mu = 0; mu < d; mu++) v[mu] = 0;
    for (;;) {
        int64_t u[ORC_MAXD];
        for (int mu = 0; mu < d; mu++) u[mu] = off[mu] + v[mu];
        if (to_buf) buf[q] = X[lin(c, u)]; else X[lin(c, u)] = buf[q];
        q++;
        int mu = 0;
        while (mu < d) { if (++v[mu] < ext[mu]) break; v[mu] = 0; mu++; }
        if (mu == d) break;
    }
}

/* Right-hand side update of Eq. (2.3a) for the Laplace form, and of the
 * d-term generalized form (term pattern of Sec. 3.1):
 *   B1 -= sum_term X2 x_1 M_{term,1} ... x_d M_{term,d}
 * where in the split mode mu the factor is the off-diagonal block
 * M_{term,mu}(off+0:k, off+k:m) and in every other mode the diagonal block
 * of the current sub-problem.  For the Laplace form only term == mu survives
 * (the identity has no off-diagonal block). */
/* Transposed operator (lower block triangular coefficients M^T): the solved
 * part is the leading one, X1 (mode-mu rows [off, off+k)), and the update goes
 * to the trailing right-hand side,
 *   B2 -= sum_term X1 x_1 M_{term,1}^T ... x_d M_{term,d}^T
 * with M_{term,mu}(off+0:k, off+k:m)^T in the split mode. */
static int rec_update(rec_ctx* r, int mu, const int64_t* off, const int64_t* ext, int64_t k, int transpose) {
    const orc_ctx* c = &r->c; int d = c->d;
    int64_t m = ext[mu];
    int64_t e2[ORC_MAXD], o2[ORC_MAXD], e1[ORC_MAXD];
    for (int q = 0; q < d; q++) { e2[q] = ext[q]; o2[q] = off[q]; e1[q] = ext[q]; }
    e2[mu] = m - k; o2[mu] = off[mu] + k; e1[mu] = k;
    /* source box (solved) and target box (right-hand side to update) */
    const int64_t* so = transpose ? off : o2;
    const int64_t* se = transpose ? e1 : e2;
    const int64_t* to = transpose ? o2 : off;
    const int64_t* te = transpose ? e2 : e1;
    int64_t Ns = prod_range(se, 0, d), Nt = prod_range(te, 0, d);
    int64_t Nmax = Ns > Nt ? Ns : Nt;
    double* xs = (double*)malloc(sizeof(double) * (size_t)Ns);
    double* t0 = (double*)malloc(sizeof(double) * (size_t)Nmax);
    double* t1 = (double*)malloc(sizeof(double) * (size_t)Nmax);
    double* bt = (double*)malloc(sizeof(double) * (size_t)Nt);
    if (!xs || !t0 || !t1 || !bt) { free(xs); free(t0); free(t1); free(bt); return -1; }
    box_io(c, r->X, so, se, xs, 1);
    box_io(c, r->X, to, te, bt, 1);
    for (int term = 0; term < d; term++) {
        if (c->C == NULL && term != mu) continue;
        int64_t cur[ORC_MAXD];
        for (int q = 0; q < d; q++) cur[q] = se[q];
        memcpy(t0, xs, sizeof(double) * (size_t)Ns);
        for (int eta = 0; eta < d; eta++) {
            const double* M;
            if (eta == term) M = c->A[eta];
            else if (c->C == NULL) continue;
            else M = c->C[eta];
            int64_t ld = c->n[eta];
            if (eta == mu) {
                /* rows of the off-diagonal block: leading indices off..off+k-1,
                 * columns: trailing indices off+k..off+m-1 */
                if (!transpose)
                    mode_product_block(d, cur, eta, M, ld, off[mu], off[mu] + k, k, 0, t0, t1);
                else
                    mode_product_block(d, cur, eta, M, ld, off[mu] + k, off[mu], m - k, 1, t0, t1);
                cur[eta] = te[mu];
            } else {
                mode_product_block(d, cur, eta, M, ld, off[eta], off[eta], ext[eta], transpose, t0, t1);
            }
            double* t = t0; t0 = t1; t1 = t;
        }
        for (int64_t q = 0; q < Nt; q++) bt[q] -= t0[q];
    }
    box_io(c, r->X, to, te, bt, 0);
    free(xs); free(t0); free(t1); free(bt);
    return 0;
}

/* transpose = 1: the same split tree for A^T (lower block triangular
 * coefficients) -- the leading part is solved first and updates the
 * trailing right-hand side (the recursion order reversed). */
static int rec_solve(rec_ctx* r, const int64_t* off, const int64_t* ext, int transpose) {
    const orc_ctx* c = &r->c; int d = c->d;
    int mu = 0;
    for (int q = 1; q < d; q++) if (ext[q] > ext[mu]) mu = q;    /* lowest mode on ties */
    if (ext[mu] <= r->nmin) return backsub_box(c, r->X, off, ext, transpose);
    int64_t m = ext[mu], k = m / 2;
    /* split rule of Alg. 2: do not cut a 2x2 block, i.e. A_mu(k+1, k) != 0 (1-based) */
    if (c->A[mu][(off[mu] + k) + c->n[mu] * (off[mu] + k - 1)] != 0.0) k += 1;
    if (k >= m) return backsub_box(c, r->X, off, ext, transpose);
    int64_t o2[ORC_MAXD], e2[ORC_MAXD], e1[ORC_MAXD];
    for (int q = 0; q < d; q++) { o2[q] = off[q]; e2[q] = ext[q]; e1[q] = ext[q]; }
    o2[mu] = off[mu] + k; e2[mu] = m - k; e1[mu] = k;
    if (!transpose) {
        int s = rec_solve(r, o2, e2, 0);                   /* trailing part X2 first (Alg. 2) */
        if (s) return s;
        if (rec_update(r, mu, off, ext, k, 0)) return -1;  /* update of B1, Eq. (2.3a) */
        return rec_solve(r, off, e1, 0);                   /* leading part X1 with the updated B1 */
    }
    int s = rec_solve(r, off, e1, 1);
    if (s) return s;
    if (rec_update(r, mu, off, ext, k, 1)) return -1;
    return rec_solve(r, o2, e2, 1);
}

/* O-B: Alg. 2 recursion with leaf size nmin (>= 1) for A (transpose = 0) or
 * A^T (transpose = 1). X: B on entry, X on exit. */
int orc_recursive(int d, const int64_t* n, const double* const* A, const double* const* C,
                  double* X, int64_t nmin, int transpose) {
    if (orc_check_structure(d, n, A) || nmin < 1) return -1;
    rec_ctx r; r.X = X; r.nmin = nmin;
    if (ctx_init(&r.c, d, n, A, C)) { ctx_free(&r.c); return -1; }
    int64_t off[ORC_MAXD] = {0};
    int s = rec_solve(&r, off, n, transpose ? 1 : 0);
    ctx_free(&r.c);
    return s;
}

/* ------------------------------------------------------------- gradients */

/* Adjoint of the solve for a scalar loss L(X):  with Lambda = A^{-T}(dL/dX),
 *   dL/dB      = Lambda
 *   dL/dA_mu   = -mask_A( Lambda_(mu) W_(mu)^T ),  W = X x_{eta != mu} C_eta
 *   dL/dC_mu   = -mask_C( sum_{nu != mu} Lambda_(mu) V_(mu)^T ),
 *                V = X x_nu A_nu x_{eta not in {mu, nu}} C_eta
 * (differentiate A(X) = B: dX = A^{-1}(dB - dA(X)), then <Lambda, dA(X)>).
 * mask_A keeps the upper triangle and the subdiagonal entries of the 2x2
 * blocks of the input A_mu; mask_C keeps the upper triangle.
 * dC may be NULL (or C NULL: Laplace form, no dC). */
static void contract_mode(int d, const int64_t* n, int mu, const double* L, const double* W, double* G, double sign) {
    int64_t Lw = prod_range(n, 0, mu), m = n[mu], R = prod_range(n, mu + 1, d);
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < m; j++) {
            double s = 0.0;
            for (int64_t r = 0; r < R; r++)
                for (int64_t l = 0; l < Lw; l++)
                    s += L[l + Lw * (i + m * r)] * W[l + Lw * (j + m * r)];
            G[i + m * j] += sign * s;
        }
}

int orc_grad(int d, const int64_t* n, const double* const* A, const double* const* C,
             const double* X, const double* Lambda, double* const* dA, double* const* dC) {
    if (orc_check_structure(d, n, A)) return -1;
    int64_t N = prod_range(n, 0, d);
    double* t0 = (double*)malloc(sizeof(double) * (size_t)N);
    double* t1 = (double*)malloc(sizeof(double) * (size_t)N);
    if (!t0 || !t1) { free(t0); free(t1); return -1; }
    for (int mu = 0; mu < d; mu++) {
        int64_t m = n[mu];
        memset(dA[mu], 0, sizeof(double) * (size_t)(m * m));
        memcpy(t0, X, sizeof(double) * (size_t)N);
        if (C != NULL)
            for (int eta = 0; eta < d; eta++) {
                if (eta == mu) continue;
                mode_product_block(d, n, eta, C[eta], n[eta], 0, 0, n[eta], 0, t0, t1);
                double* t = t0; t0 = t1; t1 = t;
            }
        contract_mode(d, n, mu, Lambda, t0, dA[mu], -1.0);
        for (int64_t i = 0; i < m; i++)
            for (int64_t j = 0; j < m; j++) {
                int keep = (i <= j) || (i == j + 1 && A[mu][i + m * j] != 0.0);
                if (!keep) dA[mu][i + m * j] = 0.0;
            }
        if (C != NULL && dC != NULL && dC[mu] != NULL) {
            memset(dC[mu], 0, sizeof(double) * (size_t)(m * m));
            for (int nu = 0; nu < d; nu++) {
                if (nu == mu) continue;
                memcpy(t0, X, sizeof(double) * (size_t)N);
                for (int eta = 0; eta < d; eta++) {
                    if (eta == mu) continue;
                    const double* M = (eta == nu) ? A[eta] : C[eta];
                    mode_product_block(d, n, eta, M, n[eta], 0, 0, n[eta], 0, t0, t1);
                    double* t = t0; t0 = t1; t1 = t;
                }
                contract_mode(d, n, mu, Lambda, t0, dC[mu], -1.0);
            }
            for (int64_t i = 0; i < m; i++)
                for (int64_t j = 0; j < i; j++) dC[mu][i + m * j] = 0.0;
        }
    }
    free(t0); free(t1);
    return 0;
}
