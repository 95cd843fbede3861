/*
 * aaomg_oracle.c -- plain, slow, FP64 CPU oracle for the all-at-once multigrid
 * method for the Poisson control problem (Takacs, "Efficient smoothers for
 * all-at-once multigrid methods for Poisson and Stokes control problems").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: it is used by the tests, by __graft_entry__.smoke() as a checker
 * and by bench.py's CPU-baseline leg.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Everything is written the direct way, in the paper's order and notation:
 *   - Section 1, eq. (mp2): Courant (P1) elements on a uniformly refined
 *     triangulation; M_k and K_k are assembled by element loops into CSR and
 *     A_k = [[M_k, K_k], [K_k, -alpha^{-1} M_k]] is built from them.
 *   - Section 2: L_k = diag(Q_k) with Q_k = blockdiag(M + alpha^{1/2} K,
 *     alpha^{-1} M + alpha^{-1/2} K).
 *   - Algorithm 1 (normal equation smoother, damped by tau) and Algorithm 2
 *     (LSGS), both maintaining the residual r = f - A x as the algorithms do.
 *   - sLSGS: one LSGS step followed by one LSGS step in reversed order.
 *   - CGS (collective point Gauss-Seidel): 2x2 block solves per node.
 *   - Section 2 multigrid: smoothing, defect, restriction by the transpose of
 *     the canonical embedding, recursive V (gamma=1) or W (gamma=2) cycle,
 *     exact solve on the coarsest grid (dense LU with partial pivoting).
 *
 * Readings of points the paper leaves open (domain, diagonal direction,
 * K = stiffness of -Lap + id, right-hand side M y_D, colour order, stopping
 * norm) are chosen by the caller through the arguments below; defaults are
 * documented where they are used.
 *
 * Floating point: IEEE double, compiled with -ffp-contract=off so that results
 * are identical on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 14

typedef struct {
    int nrows, ncols;
    int64_t nnz;
    int64_t* rowptr; /* nrows+1 */
    int* col;        /* nnz, ascending within a row */
    double* val;     /* nnz */
} ocsr;

typedef struct {
    int n;   /* cells per side; nodes (i,j), 0<=i,j<=n, index j*(n+1)+i */
    int nn;  /* (n+1)^2 nodes = unknowns per field */
    ocsr M, K, A, P; /* P: prolongation from level-1 into this level (nn x nn_coarse) */
    double* Ld;      /* diag(Q), length 2*nn */
    double* Nd;      /* N_ii = sum_j A_ij^2 / L_jj, length 2*nn (Algorithm 2, "prepare once") */
    int* order;      /* visiting order of the 2*nn unknowns for LSGS / sLSGS */
    int* corder;     /* visiting order of the nn nodes for CGS */
    double *f, *x, *r, *p; /* work vectors, length 2*nn */
} olevel;

typedef struct {
    int L;          /* finest level: h = 2^-L; coarsest level 1 (h = 1/2) */
    double alpha;
    int kvariant;   /* 0: K from (grad y, grad v) + (y, v); 1: K from (grad y, grad v) only */
    int smoother;   /* 0 NE (Alg. 1), 1 LSGS (Alg. 2), 2 sLSGS, 3 CGS */
    int nu_pre, nu_post;
    int gamma;      /* 1 V-cycle, 2 W-cycle */
    double tau;     /* NE damping */
    int lexicographic; /* 0: multicolour order, 1: natural order y_1..y_N, lambda_1..lambda_N */
    olevel lev[OR_MAXLEV + 1];
    double* clu;    /* dense LU of the coarsest A (row-major, 2nn x 2nn) */
    int* cpiv;
} ohier;

/* ------------------------------------------------------------------ CSR --- */

/* Row accumulator: every row of a P1 matrix on this mesh has at most 7 distinct
 * columns; rows are kept as short unsorted lists and merged on insertion. */
typedef struct {
    int nrows, cap;
    int* cnt;
    int* col;
    double* val;
} oacc;

static int acc_init(oacc* a, int nrows, int cap) {
    a->nrows = nrows;
    a->cap = cap;
    a->cnt = (int*)calloc((size_t)nrows, sizeof(int));
    a->col = (int*)malloc((size_t)nrows * cap * sizeof(int));
    a->val = (double*)malloc((size_t)nrows * cap * sizeof(double));
    return a->cnt && a->col && a->val ? 0 : -1;
}

static void acc_free(oacc* a) {
    free(a->cnt);
    free(a->col);
    free(a->val);
}

static int acc_add(oacc* a, int row, int col, double v) {
    int c = a->cnt[row];
    int* cols = a->col + (size_t)row * a->cap;
    double* vals = a->val + (size_t)row * a->cap;
    for (int k = 0; k < c; ++k)
        if (cols[k] == col) {
            vals[k] += v;
            return 0;
        }
    if (c == a->cap) return -1;
    cols[c] = col;
    vals[c] = v;
    a->cnt[row] = c + 1;
    return 0;
}

static int acc_to_csr(const oacc* a, int ncols, ocsr* out) {
    out->nrows = a->nrows;
    out->ncols = ncols;
    out->rowptr = (int64_t*)malloc(((size_t)a->nrows + 1) * sizeof(int64_t));
    if (!out->rowptr) return -1;
    int64_t nnz = 0;
    for (int i = 0; i < a->nrows; ++i) {
        out->rowptr[i] = nnz;
        nnz += a->cnt[i];
    }
    out->rowptr[a->nrows] = nnz;
    out->nnz = nnz;
    out->col = (int*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
    out->val = (double*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    if (!out->col || !out->val) return -1;
    for (int i = 0; i < a->nrows; ++i) {
        int c = a->cnt[i];
        const int* cols = a->col + (size_t)i * a->cap;
        const double* vals = a->val + (size_t)i * a->cap;
        int64_t base = out->rowptr[i];
        /* insertion sort by column */
        for (int k = 0; k < c; ++k) {
            int64_t pos = base + k;
            int cc = cols[k];
            double vv = vals[k];
            while (pos > base && out->col[pos - 1] > cc) {
                out->col[pos] = out->col[pos - 1];
                out->val[pos] = out->val[pos - 1];
                --pos;
            }
            out->col[pos] = cc;
            out->val[pos] = vv;
        }
    }
    return 0;
}

static void csr_free(ocsr* m) {
    free(m->rowptr);
    free(m->col);
    free(m->val);
    memset(m, 0, sizeof(*m));
}

/* y = A x */
static void csr_mv(const ocsr* A, const double* x, double* y) {
    for (int i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) s += A->val[k] * x[A->col[k]];
        y[i] = s;
    }
}

/* ------------------------------------------------------- P1 assembly --- */

/* Local P1 matrices on one triangle (section 1: Courant element).
 * mass:      |T|/12 * [[2,1,1],[1,2,1],[1,1,2]]
 * stiffness: |T| * grad(phi_a) . grad(phi_b), with the barycentric gradients
 *            grad(phi_a) = (y_b - y_c, x_c - x_b) / (2|T|), (a,b,c) cyclic. */
static void tri_local(const double px[3], const double py[3], double Ml[3][3], double Kl[3][3]) {
    double det = (px[1] - px[0]) * (py[2] - py[0]) - (px[2] - px[0]) * (py[1] - py[0]);
    double area = fabs(det) / 2.0;
    double gx[3], gy[3];
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        gx[a] = (py[b] - py[c]) / det;
        gy[a] = (px[c] - px[b]) / det;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            Ml[a][b] = area / 12.0 * (a == b ? 2.0 : 1.0);
            Kl[a][b] = area * (gx[a] * gx[b] + gy[a] * gy[b]);
        }
}

/* Assemble M and K on the uniform mesh of the unit square with n cells per
 * side, every cell split by its SW-NE diagonal ("/") into the triangles
 * {(i,j),(i+1,j),(i+1,j+1)} and {(i,j),(i+1,j+1),(i,j+1)}.  Neumann boundary:
 * every node is an unknown, nothing is eliminated.  K is the matrix of the
 * bilinear form of the state equation -Lap y + y = u, i.e. stiffness + mass
 * (kvariant 0), or the bare stiffness matrix (kvariant 1). */
static int assemble(int n, int kvariant, ocsr* M, ocsr* K) {
    int nn = (n + 1) * (n + 1);
    double h = 1.0 / n;
    oacc am, ak;
    if (acc_init(&am, nn, 7) || acc_init(&ak, nn, 7)) return -1;
    for (int cj = 0; cj < n; ++cj)
        for (int ci = 0; ci < n; ++ci) {
            int tri[2][3][2] = {{{ci, cj}, {ci + 1, cj}, {ci + 1, cj + 1}},
                                {{ci, cj}, {ci + 1, cj + 1}, {ci, cj + 1}}};
            for (int t = 0; t < 2; ++t) {
                double px[3], py[3];
                int node[3];
                for (int a = 0; a < 3; ++a) {
                    px[a] = tri[t][a][0] * h;
                    py[a] = tri[t][a][1] * h;
                    node[a] = tri[t][a][1] * (n + 1) + tri[t][a][0];
                }
                double Ml[3][3], Kl[3][3];
                tri_local(px, py, Ml, Kl);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        if (acc_add(&am, node[a], node[b], Ml[a][b])) return -1;
                        double kv = Kl[a][b] + (kvariant == 0 ? Ml[a][b] : 0.0);
                        if (acc_add(&ak, node[a], node[b], kv)) return -1;
                    }
            }
        }
    int rc = acc_to_csr(&am, nn, M) | acc_to_csr(&ak, nn, K);
    acc_free(&am);
    acc_free(&ak);
    return rc;
}

/* A = [[M, K], [K, -alpha^{-1} M]]  (eq. (mp2)), unknowns x = (y, lambda). */
static int build_A(const ocsr* M, const ocsr* K, double alpha, ocsr* A) {
    int nn = M->nrows;
    oacc aa;
    if (acc_init(&aa, 2 * nn, 14)) return -1;
    for (int i = 0; i < nn; ++i) {
        for (int64_t k = M->rowptr[i]; k < M->rowptr[i + 1]; ++k) {
            acc_add(&aa, i, M->col[k], M->val[k]);
            acc_add(&aa, nn + i, nn + M->col[k], -M->val[k] / alpha);
        }
        for (int64_t k = K->rowptr[i]; k < K->rowptr[i + 1]; ++k) {
            acc_add(&aa, i, nn + K->col[k], K->val[k]);
            acc_add(&aa, nn + i, K->col[k], K->val[k]);
        }
    }
    int rc = acc_to_csr(&aa, 2 * nn, A);
    acc_free(&aa);
    return rc;
}

static double csr_diag(const ocsr* m, int i) {
    for (int64_t k = m->rowptr[i]; k < m->rowptr[i + 1]; ++k)
        if (m->col[k] == i) return m->val[k];
    return 0.0;
}

/* L = diag(Q), Q = blockdiag(M + alpha^{1/2} K, alpha^{-1} M + alpha^{-1/2} K)  (section 2). */
static void build_L(const ocsr* M, const ocsr* K, double alpha, double* Ld) {
    int nn = M->nrows;
    for (int i = 0; i < nn; ++i) {
        double m = csr_diag(M, i), k = csr_diag(K, i);
        Ld[i] = m + sqrt(alpha) * k;
        Ld[nn + i] = m / alpha + k / sqrt(alpha);
    }
}

/* N_ii = sum_j A_ij^2 / L_jj  (Algorithm 2, "prepare once"). */
static void build_N(const ocsr* A, const double* Ld, double* Nd) {
    for (int i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) s += A->val[k] * A->val[k] / Ld[A->col[k]];
        Nd[i] = s;
    }
}

/* Prolongation I_{k-1}^k: the canonical embedding of the coarse P1 space into
 * the fine one, i.e. each fine basis coefficient is the value of the coarse
 * function at the fine node, evaluated through the coarse triangle that holds
 * the node (barycentric coordinates). */
static int build_P(int nf, ocsr* P) {
    int nc = nf / 2;
    int nnf = (nf + 1) * (nf + 1), nnc = (nc + 1) * (nc + 1);
    oacc ap;
    if (acc_init(&ap, nnf, 3)) return -1;
    for (int j = 0; j <= nf; ++j)
        for (int i = 0; i <= nf; ++i) {
            /* position in coarse cell units */
            double X = i * 0.5, Y = j * 0.5;
            int I = (int)floor(X), J = (int)floor(Y);
            if (I > nc - 1) I = nc - 1;
            if (J > nc - 1) J = nc - 1;
            double s = X - I, t = Y - J;
            int v[3];
            double w[3];
            if (s >= t) { /* lower triangle (I,J),(I+1,J),(I+1,J+1) */
                v[0] = J * (nc + 1) + I;
                v[1] = J * (nc + 1) + I + 1;
                v[2] = (J + 1) * (nc + 1) + I + 1;
                w[0] = 1.0 - s;
                w[1] = s - t;
                w[2] = t;
            } else { /* upper triangle (I,J),(I+1,J+1),(I,J+1) */
                v[0] = J * (nc + 1) + I;
                v[1] = (J + 1) * (nc + 1) + I + 1;
                v[2] = (J + 1) * (nc + 1) + I;
                w[0] = 1.0 - t;
                w[1] = s;
                w[2] = t - s;
            }
            int row = j * (nf + 1) + i;
            for (int a = 0; a < 3; ++a)
                if (w[a] != 0.0 && acc_add(&ap, row, v[a], w[a])) return -1;
        }
    int rc = acc_to_csr(&ap, nnc, P);
    acc_free(&ap);
    return rc;
}

/* ------------------------------------------------------- orderings --- */

/* Multicolour order: colour(i,j) = (i + 2j) mod 7, a distance-2 colouring of
 * the "/" lattice (two nodes of equal colour never share a neighbour, so the
 * LSGS updates within one colour do not interact).  The y unknowns are visited
 * first, then the lambda unknowns (the block order of x in eq. (mp2)); within
 * a field the colours are visited in the sequence 0,6,5,4,3,2,1 and the nodes
 * of one colour by increasing index. */
static const int COLOUR_SEQ[7] = {0, 6, 5, 4, 3, 2, 1};

static void build_order(int n, int lexicographic, int* order) {
    int nn = (n + 1) * (n + 1);
    int pos = 0;
    if (lexicographic) {
        for (int u = 0; u < 2 * nn; ++u) order[u] = u;
        return;
    }
    for (int field = 0; field < 2; ++field)
        for (int s = 0; s < 7; ++s)
            for (int j = 0; j <= n; ++j)
                for (int i = 0; i <= n; ++i)
                    if ((i + 2 * j) % 7 == COLOUR_SEQ[s]) order[pos++] = field * nn + j * (n + 1) + i;
}

/* CGS visits nodes; A couples nodes at graph distance 1 only, so the colouring
 * (i + j) mod 3 separates the 2x2 block updates of one colour. */
static void build_corder(int n, int lexicographic, int* corder) {
    int pos = 0;
    if (lexicographic) {
        for (int u = 0; u < (n + 1) * (n + 1); ++u) corder[u] = u;
        return;
    }
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i)
                if ((i + j) % 3 == c) corder[pos++] = j * (n + 1) + i;
}

/* ------------------------------------------------------- hierarchy --- */

static void level_free(olevel* l) {
    csr_free(&l->M);
    csr_free(&l->K);
    csr_free(&l->A);
    csr_free(&l->P);
    free(l->Ld);
    free(l->Nd);
    free(l->order);
    free(l->corder);
    free(l->f);
    free(l->x);
    free(l->r);
    free(l->p);
    memset(l, 0, sizeof(*l));
}

static int lu_factor(int m, double* a, int* piv);

void or_destroy(ohier* H) {
    if (!H) return;
    for (int k = 1; k <= OR_MAXLEV; ++k) level_free(&H->lev[k]);
    free(H->clu);
    free(H->cpiv);
    free(H);
}

ohier* or_create(int L, double alpha, int kvariant, int smoother, int nu_pre, int nu_post, int gamma, double tau,
                 int lexicographic) {
    if (L < 1 || L > OR_MAXLEV || !(alpha > 0.0)) return NULL;
    ohier* H = (ohier*)calloc(1, sizeof(ohier));
    if (!H) return NULL;
    H->L = L;
    H->alpha = alpha;
    H->kvariant = kvariant;
    H->smoother = smoother;
    H->nu_pre = nu_pre;
    H->nu_post = nu_post;
    H->gamma = gamma;
    H->tau = tau;
    H->lexicographic = lexicographic;
    for (int k = 1; k <= L; ++k) {
        olevel* l = &H->lev[k];
        l->n = 1 << k;
        l->nn = (l->n + 1) * (l->n + 1);
        size_t n2 = 2 * (size_t)l->nn;
        if (assemble(l->n, kvariant, &l->M, &l->K) || build_A(&l->M, &l->K, alpha, &l->A)) goto fail;
        l->Ld = (double*)malloc(n2 * sizeof(double));
        l->Nd = (double*)malloc(n2 * sizeof(double));
        l->order = (int*)malloc(n2 * sizeof(int));
        l->corder = (int*)malloc((size_t)l->nn * sizeof(int));
        l->f = (double*)calloc(n2, sizeof(double));
        l->x = (double*)calloc(n2, sizeof(double));
        l->r = (double*)calloc(n2, sizeof(double));
        l->p = (double*)calloc(n2, sizeof(double));
        if (!l->Ld || !l->Nd || !l->order || !l->corder || !l->f || !l->x || !l->r || !l->p) goto fail;
        build_L(&l->M, &l->K, alpha, l->Ld);
        build_N(&l->A, l->Ld, l->Nd);
        build_order(l->n, lexicographic, l->order);
        build_corder(l->n, lexicographic, l->corder);
        if (k > 1 && build_P(l->n, &l->P)) goto fail;
    }
    {
        /* coarsest level: dense LU of A_1 */
        olevel* c = &H->lev[1];
        int m = 2 * c->nn;
        H->clu = (double*)calloc((size_t)m * m, sizeof(double));
        H->cpiv = (int*)malloc((size_t)m * sizeof(int));
        if (!H->clu || !H->cpiv) goto fail;
        for (int i = 0; i < m; ++i)
            for (int64_t k = c->A.rowptr[i]; k < c->A.rowptr[i + 1]; ++k) H->clu[(size_t)i * m + c->A.col[k]] = c->A.val[k];
        if (lu_factor(m, H->clu, H->cpiv)) goto fail;
    }
    return H;
fail:
    or_destroy(H);
    return NULL;
}

int or_nnodes(const ohier* H, int level) { return H->lev[level].nn; }

int64_t or_csr_nnz(const ohier* H, int level, int which) {
    const olevel* l = &H->lev[level];
    const ocsr* m = which == 0 ? &l->M : which == 1 ? &l->K : which == 2 ? &l->A : &l->P;
    return m->nnz;
}

int or_csr_shape(const ohier* H, int level, int which, int* nrows, int* ncols) {
    const olevel* l = &H->lev[level];
    const ocsr* m = which == 0 ? &l->M : which == 1 ? &l->K : which == 2 ? &l->A : &l->P;
    *nrows = m->nrows;
    *ncols = m->ncols;
    return 0;
}

void or_csr_export(const ohier* H, int level, int which, int64_t* rowptr, int* col, double* val) {
    const olevel* l = &H->lev[level];
    const ocsr* m = which == 0 ? &l->M : which == 1 ? &l->K : which == 2 ? &l->A : &l->P;
    memcpy(rowptr, m->rowptr, ((size_t)m->nrows + 1) * sizeof(int64_t));
    memcpy(col, m->col, (size_t)m->nnz * sizeof(int));
    memcpy(val, m->val, (size_t)m->nnz * sizeof(double));
}

void or_ldiag(const ohier* H, int level, double* out) {
    memcpy(out, H->lev[level].Ld, 2 * (size_t)H->lev[level].nn * sizeof(double));
}
void or_ndiag(const ohier* H, int level, double* out) {
    memcpy(out, H->lev[level].Nd, 2 * (size_t)H->lev[level].nn * sizeof(double));
}
void or_order(const ohier* H, int level, int* out) {
    memcpy(out, H->lev[level].order, 2 * (size_t)H->lev[level].nn * sizeof(int));
}

/* ------------------------------------------------------- basic ops --- */

/* right-hand side of eq. (mp2): f = (M y_D, 0) with y_D the nodal values of the
 * desired state (from the optimality condition M y + K lambda = M y_D). */
void or_rhs(const ohier* H, const double* yD, double* f) {
    const olevel* l = &H->lev[H->L];
    csr_mv(&l->M, yD, f);
    for (int i = 0; i < l->nn; ++i) f[l->nn + i] = 0.0;
}

/* r = f - A x */
void or_residual(const ohier* H, int level, const double* f, const double* x, double* r) {
    const olevel* l = &H->lev[level];
    csr_mv(&l->A, x, r);
    for (int i = 0; i < 2 * l->nn; ++i) r[i] = f[i] - r[i];
}

/* ||v||_{L^{-1}} = (v^T L^{-1} v)^{1/2}: the norm of a residual, dual to the
 * norm ||.||_L in which the paper measures errors. */
double or_norm_Linv(const ohier* H, int level, const double* v) {
    const olevel* l = &H->lev[level];
    double s = 0.0;
    for (int i = 0; i < 2 * l->nn; ++i) s += v[i] * v[i] / l->Ld[i];
    return sqrt(s);
}

/* ||v||_L = (v^T L v)^{1/2} (section 2, the norm of the smoothing property). */
double or_norm_L(const ohier* H, int level, const double* v) {
    const olevel* l = &H->lev[level];
    double s = 0.0;
    for (int i = 0; i < 2 * l->nn; ++i) s += v[i] * v[i] * l->Ld[i];
    return sqrt(s);
}

/* --------------------------------------------------------- smoothers --- */
/* The matrix A is symmetric (it is assembled from symmetric M and K), so the
 * column A_{:,i} that Algorithms 1 and 2 walk equals the row A_{i,:}. */

/* Algorithm 1: one normal-equation step, x <- x + tau L^{-1} A^T L^{-1} r,
 * with the residual r = f - A x updated alongside. */
static void ne_step(olevel* l, double tau, double* x, double* r) {
    const ocsr* A = &l->A;
    int m = 2 * l->nn;
    double* p = l->p;
    for (int i = 0; i < m; ++i) {
        double q = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) q += A->val[k] / l->Ld[A->col[k]] * r[A->col[k]];
        p[i] = tau * q / l->Ld[i];
    }
    for (int i = 0; i < m; ++i) {
        x[i] += p[i];
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) r[A->col[k]] -= A->val[k] * p[i];
    }
}

/* Algorithm 2: one LSGS step, Gauss-Seidel on the normal equation
 * N x = A^T L^{-1} f with N = A^T L^{-1} A, in the order `order` (reversed when
 * `reverse` is set, which gives the second half of an sLSGS step). */
static void lsgs_step(olevel* l, const int* order, int reverse, double* x, double* r) {
    const ocsr* A = &l->A;
    int m = 2 * l->nn;
    for (int s = 0; s < m; ++s) {
        int i = order[reverse ? m - 1 - s : s];
        double q = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) q += A->val[k] / l->Ld[A->col[k]] * r[A->col[k]];
        double p = q / l->Nd[i];
        x[i] += p;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) r[A->col[k]] -= A->val[k] * p;
    }
}

/* Collective Gauss-Seidel: for each node i, solve the 2x2 system
 * [[M_ii, K_ii], [K_ii, -alpha^{-1} M_ii]] (dy, dlambda) = (r_y_i, r_lambda_i)
 * and add the update, keeping r current. */
static void cgs_step(olevel* l, const int* corder, double alpha, double* x, double* r) {
    const ocsr* A = &l->A;
    int nn = l->nn;
    for (int s = 0; s < nn; ++s) {
        int i = corder[s];
        double m = csr_diag(&l->M, i), k = csr_diag(&l->K, i);
        double a11 = m, a12 = k, a21 = k, a22 = -m / alpha;
        double det = a11 * a22 - a12 * a21;
        double b1 = r[i], b2 = r[nn + i];
        double dy = (a22 * b1 - a12 * b2) / det;
        double dl = (a11 * b2 - a21 * b1) / det;
        x[i] += dy;
        x[nn + i] += dl;
        for (int64_t q = A->rowptr[i]; q < A->rowptr[i + 1]; ++q) r[A->col[q]] -= A->val[q] * dy;
        for (int64_t q = A->rowptr[nn + i]; q < A->rowptr[nn + i + 1]; ++q) r[A->col[q]] -= A->val[q] * dl;
    }
}

/* `steps` smoothing steps x^{(0,m)} = x^{(0,m-1)} + Ahat^{-1}(f - A x^{(0,m-1)})
 * with the configured smoother; the residual is formed once and then carried
 * along by the algorithms. */
void or_smooth(ohier* H, int level, const double* f, double* x, int steps) {
    olevel* l = &H->lev[level];
    or_residual(H, level, f, x, l->r);
    for (int m = 0; m < steps; ++m) {
        switch (H->smoother) {
        case 0: ne_step(l, H->tau, x, l->r); break;
        case 1: lsgs_step(l, l->order, 0, x, l->r); break;
        case 2:
            lsgs_step(l, l->order, 0, x, l->r);
            lsgs_step(l, l->order, 1, x, l->r);
            break;
        default: cgs_step(l, l->corder, H->alpha, x, l->r); break;
        }
    }
}

/* ------------------------------------------------------- transfers --- */

/* restriction I_k^{k-1} = (I_{k-1}^k)^T, applied to both fields: rc = P^T rf */
void or_restrict(const ohier* H, int level, const double* rf, double* rc) {
    const olevel* l = &H->lev[level];
    const ocsr* P = &l->P;
    int nc = P->ncols, nf = P->nrows;
    for (int i = 0; i < 2 * nc; ++i) rc[i] = 0.0;
    for (int field = 0; field < 2; ++field)
        for (int i = 0; i < nf; ++i)
            for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) rc[field * nc + P->col[k]] += P->val[k] * rf[field * nf + i];
}

/* xf += I_{k-1}^k xc on both fields */
void or_prolong_add(const ohier* H, int level, const double* xc, double* xf) {
    const olevel* l = &H->lev[level];
    const ocsr* P = &l->P;
    int nc = P->ncols, nf = P->nrows;
    for (int field = 0; field < 2; ++field)
        for (int i = 0; i < nf; ++i) {
            double s = 0.0;
            for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) s += P->val[k] * xc[field * nc + P->col[k]];
            xf[field * nf + i] += s;
        }
}

/* ------------------------------------------------------- coarse solve --- */

/* LU with partial pivoting, row-major, in place. */
static int lu_factor(int m, double* a, int* piv) {
    for (int k = 0; k < m; ++k) {
        int p = k;
        double best = fabs(a[(size_t)k * m + k]);
        for (int i = k + 1; i < m; ++i)
            if (fabs(a[(size_t)i * m + k]) > best) {
                best = fabs(a[(size_t)i * m + k]);
                p = i;
            }
        if (best == 0.0) return -1;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < m; ++j) {
                double t = a[(size_t)k * m + j];
                a[(size_t)k * m + j] = a[(size_t)p * m + j];
                a[(size_t)p * m + j] = t;
            }
        for (int i = k + 1; i < m; ++i) {
            double f = a[(size_t)i * m + k] / a[(size_t)k * m + k];
            a[(size_t)i * m + k] = f;
            for (int j = k + 1; j < m; ++j) a[(size_t)i * m + j] -= f * a[(size_t)k * m + j];
        }
    }
    return 0;
}

static void lu_solve(int m, const double* a, const int* piv, double* b) {
    for (int k = 0; k < m; ++k)
        if (piv[k] != k) {
            double t = b[k];
            b[k] = b[piv[k]];
            b[piv[k]] = t;
        }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * m + j] * b[j];
    for (int i = m - 1; i >= 0; --i) {
        for (int j = i + 1; j < m; ++j) b[i] -= a[(size_t)i * m + j] * b[j];
        b[i] /= a[(size_t)i * m + i];
    }
}

/* exact solve on the coarsest grid (level 1, h = 1/2, 18 unknowns) */
void or_coarse_solve(const ohier* H, const double* f, double* x) {
    int m = 2 * H->lev[1].nn;
    for (int i = 0; i < m; ++i) x[i] = f[i];
    lu_solve(m, H->clu, H->cpiv, x);
}

/* ------------------------------------------------------- multigrid --- */

/* One multigrid iteration on level k (section 2): nu_pre smoothing steps, the
 * defect restricted to level k-1, gamma recursive iterations on the coarse
 * problem from a zero initial guess (exact solve on level 1), prolongation and
 * correction, nu_post smoothing steps with the same smoother. */
static void cycle_rec(ohier* H, int k, const double* f, double* x) {
    if (k == 1) {
        or_coarse_solve(H, f, x);
        return;
    }
    olevel* l = &H->lev[k];
    olevel* c = &H->lev[k - 1];
    if (H->nu_pre > 0) or_smooth(H, k, f, x, H->nu_pre);
    or_residual(H, k, f, x, l->r);
    or_restrict(H, k, l->r, c->f);
    for (int i = 0; i < 2 * c->nn; ++i) c->x[i] = 0.0;
    for (int g = 0; g < H->gamma; ++g) cycle_rec(H, k - 1, c->f, c->x);
    or_prolong_add(H, k, c->x, x);
    if (H->nu_post > 0) or_smooth(H, k, f, x, H->nu_post);
}

void or_cycle(ohier* H, int level, const double* f, double* x) { cycle_rec(H, level, f, x); }

/* Iterate cycles on the finest level until ||f - A x||_{L^{-1}} <= tol *
 * ||f||_{L^{-1}} (relative residual in the dual norm of ||.||_L) or max_iter
 * cycles.  Returns the number of cycles; relres gets the final relative
 * residual and history[0..iters] (if non-NULL) every relative residual seen. */
int or_solve(ohier* H, const double* f, double* x, double tol, int max_iter, double* relres, double* history) {
    int L = H->L;
    olevel* l = &H->lev[L];
    double fn = or_norm_Linv(H, L, f);
    if (fn == 0.0) fn = 1.0;
    int it = 0;
    double rr;
    for (;;) {
        or_residual(H, L, f, x, l->r);
        rr = or_norm_Linv(H, L, l->r) / fn;
        if (history) history[it] = rr;
        if (rr <= tol || it >= max_iter || !(rr == rr)) break;
        cycle_rec(H, L, f, x);
        ++it;
    }
    if (relres) *relres = rr;
    return it;
}

/* The experiment protocol of section 3: zero right-hand side, a given (random)
 * initial guess x0, iterate until the error ||x - 0||_L has dropped by the
 * factor `reduction`.  Returns the number of iterations (or -1 beyond
 * max_iter); x0 is overwritten by the last iterate. */
int or_protocol_iterations(ohier* H, double* x0, double reduction, int max_iter) {
    int L = H->L;
    olevel* l = &H->lev[L];
    double* zero = (double*)calloc(2 * (size_t)l->nn, sizeof(double));
    if (!zero) return -2;
    double e0 = or_norm_L(H, L, x0);
    int it = 0;
    while (or_norm_L(H, L, x0) > reduction * e0) {
        if (it >= max_iter) {
            it = -1;
            break;
        }
        cycle_rec(H, L, zero, x0);
        ++it;
    }
    free(zero);
    return it;
}
