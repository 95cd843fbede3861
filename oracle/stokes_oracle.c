/*
 * stokes_oracle.c -- plain, slow, FP64 CPU oracle for the all-at-once multigrid
 * method applied to the Stokes control problem (Takacs, "Efficient smoothers
 * for all-at-once multigrid methods for Poisson and Stokes control problems",
 * section 1, second model problem; sections 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file: it is used by the tests and by bench.py's CPU legs.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Written the direct way, in the paper's order and notation:
 *   - Section 1, eq. (mp3): Taylor-Hood elements on the uniformly refined
 *     triangulation of the unit square (every cell split by its SW-NE
 *     diagonal): continuous P2 velocity v and adjoint velocity lambda, both
 *     zero on the boundary (v = 0 on the boundary; the adjoint inherits it),
 *     continuous P1 pressure p and adjoint pressure mu.  M_k and K_k are the
 *     vector P2 mass and stiffness matrices (one block per component), D_k the
 *     discrete divergence, (D v)_q = -int psi_q div v, so that D^T is the
 *     discrete gradient.  Element matrices come from exact integration of
 *     barycentric monomials,
 *         int_T l0^a l1^b l2^c = 2 |T| a! b! c! / (a + b + c + 2)!.
 *     A_k = [[M, 0, K, D^T], [0, 0, D, 0], [K, D^T, -alpha^{-1} M, 0],
 *            [D, 0, 0, 0]]  for x = (v, p, lambda, mu).
 *   - Section 2: L_k = blockdiag(W^, P^, alpha^{-1} W^, alpha^{-1} P^) with
 *     W^ = diag(M + alpha^{1/2} K) and P^ = alpha diag(D W^{-1} D^T).
 *   - Algorithm 1 (normal equation smoother, damped by tau), Algorithm 2
 *     (LSGS), sLSGS (an LSGS step followed by one in reversed order), all on
 *     the residual r = f - A x carried along as the algorithms do.
 *   - Section 2 multigrid: smoothing, defect, restriction by the transposes of
 *     the canonical embeddings of the nested P2 and P1 spaces, gamma recursive
 *     iterations (V or W), exact solve on the coarsest grid (h = 1/2).
 *   - Section 3 protocol: zero right-hand side, random start, error reduced by
 *     a given factor in ||.||_L.
 *
 * Readings where the paper is silent:
 *   - p and mu are determined up to constants only: A_k has the kernel spanned
 *     by (0, 1, 0, 0) and (0, 0, 0, 1) (D^T applied to a constant vanishes for
 *     velocities that are zero on the boundary).  The paper fixes int p = 0.
 *     Every correction of the iteration depends on the residual only, which
 *     does not see these components, so the iteration is run as it is; the
 *     coarsest solve returns the solution with int p = int mu = 0 (a bordered
 *     system), and errors are measured after removing the means of p and mu
 *     (sto_normalize).
 *   - the order of the unknowns in Algorithm 2: the natural order of x
 *     (lexicographic = 1), or a multicolour order in which the unknowns of one
 *     colour have disjoint rows in A (the order a parallel implementation can
 *     follow): block by block (v_1, v_2, p, lambda_1, lambda_2, mu); on the P2
 *     half-step grid (node (a, b) at (a h/2, b h/2)) colour (a + 7 b) mod 19,
 *     on the P1 vertices (i, j) colour (i + 2 j) mod 7; colours in increasing
 *     order, the nodes of one colour by increasing index.
 *   - right-hand side f = (M v_D, 0, 0, 0) with v_D given at every P2 node
 *     (boundary nodes included, weighted by the full P2 mass matrix).
 *
 * Floating point: IEEE double, compiled with -ffp-contract=off; duplicate
 * matrix entries are summed in insertion order, so results do not depend on
 * the host's sort routine.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ST_MAXLEV 11
#define VCOL 19 /* colours of the P2 half-step grid: (a + 7 b) mod 19 */
#define PCOL 7  /* colours of the P1 vertices: (i + 2 j) mod 7 */

typedef struct {
    int nrows, ncols;
    int64_t nnz;
    int64_t* rowptr;
    int* col;
    double* val;
} scsr;

/* ---------------------------------------------------- triplets -> CSR --- */

typedef struct {
    int row, col;
    int64_t seq;
    double val;
} strip3;

typedef struct {
    strip3* t;
    int64_t n, cap;
} scoo;

static int coo_add(scoo* c, int row, int col, double v) {
    if (c->n == c->cap) {
        int64_t cap = c->cap ? 2 * c->cap : 1024;
        strip3* t = (strip3*)realloc(c->t, (size_t)cap * sizeof(strip3));
        if (!t) return -1;
        c->t = t;
        c->cap = cap;
    }
    c->t[c->n].row = row;
    c->t[c->n].col = col;
    c->t[c->n].seq = c->n;
    c->t[c->n].val = v;
    ++c->n;
    return 0;
}

static int trip_cmp(const void* a, const void* b) {
    const strip3* x = (const strip3*)a;
    const strip3* y = (const strip3*)b;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return x->seq < y->seq ? -1 : (x->seq > y->seq);
}

/* sorted by (row, col, insertion), duplicates summed in insertion order;
 * explicit zeros are kept (the structure is that of the element loops) */
static int coo_to_csr(scoo* c, int nrows, int ncols, scsr* m) {
    qsort(c->t, (size_t)c->n, sizeof(strip3), trip_cmp);
    m->nrows = nrows;
    m->ncols = ncols;
    m->rowptr = (int64_t*)calloc((size_t)nrows + 1, sizeof(int64_t));
    m->col = (int*)malloc((size_t)(c->n ? c->n : 1) * sizeof(int));
    m->val = (double*)malloc((size_t)(c->n ? c->n : 1) * sizeof(double));
    if (!m->rowptr || !m->col || !m->val) return -1;
    int64_t k = 0;
    for (int64_t s = 0; s < c->n; ++s) {
        if (k > 0 && m->col[k - 1] == c->t[s].col && s > 0 && c->t[s - 1].row == c->t[s].row) {
            m->val[k - 1] += c->t[s].val;
            continue;
        }
        m->col[k] = c->t[s].col;
        m->val[k] = c->t[s].val;
        m->rowptr[c->t[s].row + 1] = k + 1;
        ++k;
    }
    for (int i = 0; i < nrows; ++i)
        if (m->rowptr[i + 1] < m->rowptr[i]) m->rowptr[i + 1] = m->rowptr[i];
    m->nnz = k;
    free(c->t);
    c->t = NULL;
    c->n = c->cap = 0;
    return 0;
}

static void csr_free(scsr* m) {
    free(m->rowptr);
    free(m->col);
    free(m->val);
    memset(m, 0, sizeof(*m));
}

static double csr_entry(const scsr* m, int i, int j) {
    for (int64_t k = m->rowptr[i]; k < m->rowptr[i + 1]; ++k)
        if (m->col[k] == j) return m->val[k];
    return 0.0;
}

/* y = A x */
static void csr_mv(const scsr* A, const double* x, double* y) {
    for (int i = 0; i < A->nrows; ++i) {
        double s = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) s += A->val[k] * x[A->col[k]];
        y[i] = s;
    }
}

/* ------------------------------------- barycentric polynomials, exact --- */
/* A polynomial of degree <= 4 in each of the barycentric coordinates l0, l1,
 * l2 of a triangle, coefficients c[a][b][c] of l0^a l1^b l2^c. */
typedef struct {
    double c[5][5][5];
} bpoly;

static void bp_zero(bpoly* p) { memset(p, 0, sizeof(*p)); }

static void bp_mono(bpoly* p, double coef, int a, int b, int c) {
    bp_zero(p);
    p->c[a][b][c] = coef;
}

static void bp_add_mono(bpoly* p, double coef, int a, int b, int c) { p->c[a][b][c] += coef; }

/* product, degrees of the factors summing to at most 4 per variable */
static void bp_mul(const bpoly* x, const bpoly* y, bpoly* out) {
    bp_zero(out);
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c) {
                double u = x->c[a][b][c];
                if (u == 0.0) continue;
                for (int d = 0; a + d < 5; ++d)
                    for (int e = 0; b + e < 5; ++e)
                        for (int f = 0; c + f < 5; ++f) {
                            double v = y->c[d][e][f];
                            if (v != 0.0) out->c[a + d][b + e][c + f] += u * v;
                        }
            }
}

static double fact(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

/* int_T p dx = sum c_abc 2 |T| a! b! c! / (a + b + c + 2)! */
static double bp_int(const bpoly* p, double area) {
    double s = 0.0;
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b)
            for (int c = 0; c < 5; ++c)
                if (p->c[a][b][c] != 0.0) s += p->c[a][b][c] * 2.0 * area * fact(a) * fact(b) * fact(c) / fact(a + b + c + 2);
    return s;
}

/* local P2 nodes: 0, 1, 2 the vertices, 3 = mid(0,1), 4 = mid(1,2), 5 = mid(2,0) */
static const int EDGE[3][2] = {{0, 1}, {1, 2}, {2, 0}};

static void mono_of(int v, int deg, int e[3]) {
    e[0] = e[1] = e[2] = 0;
    e[v] = deg;
}

/* P2 basis: vertex a: l_a (2 l_a - 1); edge (a, b): 4 l_a l_b */
static void p2_basis(int s, bpoly* p) {
    bp_zero(p);
    int e[3];
    if (s < 3) {
        mono_of(s, 2, e);
        bp_add_mono(p, 2.0, e[0], e[1], e[2]);
        mono_of(s, 1, e);
        bp_add_mono(p, -1.0, e[0], e[1], e[2]);
    } else {
        int a = EDGE[s - 3][0], b = EDGE[s - 3][1];
        int m[3] = {0, 0, 0};
        m[a] += 1;
        m[b] += 1;
        bp_add_mono(p, 4.0, m[0], m[1], m[2]);
    }
}

/* d(basis s) / d l_k, treating the l's as independent (chain rule:
 * grad phi = sum_k (d phi / d l_k) grad l_k) */
static void p2_dbasis(int s, int k, bpoly* p) {
    bp_zero(p);
    int e[3];
    if (s < 3) {
        if (k == s) {
            mono_of(s, 1, e);
            bp_add_mono(p, 4.0, e[0], e[1], e[2]);
            bp_add_mono(p, -1.0, 0, 0, 0);
        }
    } else {
        int a = EDGE[s - 3][0], b = EDGE[s - 3][1];
        if (k == a) {
            mono_of(b, 1, e);
            bp_add_mono(p, 4.0, e[0], e[1], e[2]);
        } else if (k == b) {
            mono_of(a, 1, e);
            bp_add_mono(p, 4.0, e[0], e[1], e[2]);
        }
    }
}

/* Local matrices of one triangle (vertices counterclockwise):
 *   Ml[s][t] = int phi_s phi_t,  Kl[s][t] = int grad phi_s . grad phi_t,
 *   Dl[c][q][t] = -int l_q d_c phi_t   (c = 0: x, 1: y; q a vertex). */
static void p2_local(const double px[3], const double py[3], double Ml[6][6], double Kl[6][6], double Dl[2][3][6]) {
    double det = (px[1] - px[0]) * (py[2] - py[0]) - (px[2] - px[0]) * (py[1] - py[0]);
    double area = fabs(det) / 2.0;
    double gx[3], gy[3]; /* grad l_a = (y_b - y_c, x_c - x_b) / det, (a, b, c) cyclic */
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        gx[a] = (py[b] - py[c]) / det;
        gy[a] = (px[c] - px[b]) / det;
    }
    bpoly phi[6], dphi[6][3], prod;
    for (int s = 0; s < 6; ++s) {
        p2_basis(s, &phi[s]);
        for (int k = 0; k < 3; ++k) p2_dbasis(s, k, &dphi[s][k]);
    }
    for (int s = 0; s < 6; ++s)
        for (int t = 0; t < 6; ++t) {
            bp_mul(&phi[s], &phi[t], &prod);
            Ml[s][t] = bp_int(&prod, area);
            double k = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    bp_mul(&dphi[s][a], &dphi[t][b], &prod);
                    k += (gx[a] * gx[b] + gy[a] * gy[b]) * bp_int(&prod, area);
                }
            Kl[s][t] = k;
        }
    for (int q = 0; q < 3; ++q) {
        bpoly lq;
        int e[3];
        mono_of(q, 1, e);
        bp_mono(&lq, 1.0, e[0], e[1], e[2]);
        for (int t = 0; t < 6; ++t) {
            double dx = 0.0, dy = 0.0;
            for (int k = 0; k < 3; ++k) {
                bp_mul(&lq, &dphi[t][k], &prod);
                double v = bp_int(&prod, area);
                dx += gx[k] * v;
                dy += gy[k] * v;
            }
            Dl[0][q][t] = -dx;
            Dl[1][q][t] = -dy;
        }
    }
}

/* ------------------------------------------------------------ levels --- */

typedef struct {
    int n;  /* cells per side, h = 1/n */
    int ng; /* P2 half-step grid nodes per side, 2n + 1 */
    int nv; /* interior P2 nodes (2n - 1)^2: unknowns per velocity component */
    int np; /* P1 vertices (n + 1)^2 */
    int m;  /* unknowns 4 nv + 2 np */
    scsr Mf, Kf, Dxf, Dyf; /* over all ng^2 P2 nodes (D: np x ng^2) */
    scsr M, K, Dx, Dy;     /* interior P2 nodes only */
    scsr A;
    scsr P2, P1; /* canonical embeddings from level - 1 (interior P2 nodes; all vertices) */
    double* Ld;
    double* Nd; /* N_ii = sum_j A_ji^2 / L_jj (Algorithm 2, "prepare once") */
    double* w;  /* int psi_q over the domain (the P1 functional of int p) */
    int* order;
    double *f, *x, *r, *p;
} slevel;

typedef struct {
    int L;
    double alpha;
    int smoother; /* 0 NE (Alg. 1), 1 LSGS (Alg. 2), 2 sLSGS */
    int nu_pre, nu_post, gamma;
    double tau;
    int lexicographic;
    slevel lev[ST_MAXLEV + 1];
    int cm;       /* bordered coarsest system size m_1 + 2 */
    double* clu;  /* its dense LU */
    int* cpiv;
} shier;

/* interior P2 node (a, b) of the half-step grid -> velocity index, or -1 */
static int vidx(const slevel* l, int a, int b) {
    if (a < 1 || b < 1 || a > l->ng - 2 || b > l->ng - 2) return -1;
    return (b - 1) * (l->ng - 2) + (a - 1);
}

/* block offsets in x = (v_1, v_2, p, lambda_1, lambda_2, mu) */
static int off_v(const slevel* l, int c) { return c * l->nv; }
static int off_p(const slevel* l) { return 2 * l->nv; }
static int off_l(const slevel* l, int c) { return 2 * l->nv + l->np + c * l->nv; }
static int off_mu(const slevel* l) { return 4 * l->nv + l->np; }

/* Element loops over the 2 n^2 triangles {(i,j),(i+1,j),(i+1,j+1)} and
 * {(i,j),(i+1,j+1),(i,j+1)}; every triangle of one shape is a translate of the
 * others, so its local matrices are computed once per shape. */
static int assemble(slevel* l) {
    int n = l->n, ng = l->ng;
    double h = 1.0 / n;
    static const int TV[2][3][2] = {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}};
    double Ml[2][6][6], Kl[2][6][6], Dl[2][2][3][6];
    for (int t = 0; t < 2; ++t) {
        double px[3], py[3];
        for (int a = 0; a < 3; ++a) {
            px[a] = TV[t][a][0] * h;
            py[a] = TV[t][a][1] * h;
        }
        p2_local(px, py, Ml[t], Kl[t], Dl[t]);
    }
    scoo cm = {0}, ck = {0}, cdx = {0}, cdy = {0};
    l->w = (double*)calloc((size_t)l->np, sizeof(double));
    if (!l->w) return -1;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            for (int t = 0; t < 2; ++t) {
                int va[3], vb[3], g[6], q[3];
                for (int a = 0; a < 3; ++a) {
                    va[a] = 2 * (i + TV[t][a][0]);
                    vb[a] = 2 * (j + TV[t][a][1]);
                    g[a] = vb[a] * ng + va[a];
                    q[a] = (j + TV[t][a][1]) * (n + 1) + (i + TV[t][a][0]);
                    l->w[q[a]] += h * h / 2.0 / 3.0;
                }
                for (int e = 0; e < 3; ++e) {
                    int a = EDGE[e][0], b = EDGE[e][1];
                    g[3 + e] = ((vb[a] + vb[b]) / 2) * ng + (va[a] + va[b]) / 2;
                }
                for (int s = 0; s < 6; ++s)
                    for (int u = 0; u < 6; ++u) {
                        if (coo_add(&cm, g[s], g[u], Ml[t][s][u]) || coo_add(&ck, g[s], g[u], Kl[t][s][u])) return -1;
                    }
                for (int a = 0; a < 3; ++a)
                    for (int u = 0; u < 6; ++u) {
                        if (coo_add(&cdx, q[a], g[u], Dl[t][0][a][u]) || coo_add(&cdy, q[a], g[u], Dl[t][1][a][u]))
                            return -1;
                    }
            }
    if (coo_to_csr(&cm, ng * ng, ng * ng, &l->Mf) || coo_to_csr(&ck, ng * ng, ng * ng, &l->Kf) ||
        coo_to_csr(&cdx, l->np, ng * ng, &l->Dxf) || coo_to_csr(&cdy, l->np, ng * ng, &l->Dyf))
        return -1;
    /* restriction to the interior P2 nodes (v = lambda = 0 on the boundary) */
    scoo rm = {0}, rk = {0}, rdx = {0}, rdy = {0};
    for (int gi = 0; gi < ng * ng; ++gi) {
        int vi = vidx(l, gi % ng, gi / ng);
        if (vi < 0) continue;
        for (int64_t k = l->Mf.rowptr[gi]; k < l->Mf.rowptr[gi + 1]; ++k) {
            int gj = l->Mf.col[k], vj = vidx(l, gj % ng, gj / ng);
            if (vj >= 0 && coo_add(&rm, vi, vj, l->Mf.val[k])) return -1;
        }
        for (int64_t k = l->Kf.rowptr[gi]; k < l->Kf.rowptr[gi + 1]; ++k) {
            int gj = l->Kf.col[k], vj = vidx(l, gj % ng, gj / ng);
            if (vj >= 0 && coo_add(&rk, vi, vj, l->Kf.val[k])) return -1;
        }
    }
    for (int q = 0; q < l->np; ++q) {
        for (int64_t k = l->Dxf.rowptr[q]; k < l->Dxf.rowptr[q + 1]; ++k) {
            int gj = l->Dxf.col[k], vj = vidx(l, gj % ng, gj / ng);
            if (vj >= 0 && coo_add(&rdx, q, vj, l->Dxf.val[k])) return -1;
        }
        for (int64_t k = l->Dyf.rowptr[q]; k < l->Dyf.rowptr[q + 1]; ++k) {
            int gj = l->Dyf.col[k], vj = vidx(l, gj % ng, gj / ng);
            if (vj >= 0 && coo_add(&rdy, q, vj, l->Dyf.val[k])) return -1;
        }
    }
    if (coo_to_csr(&rm, l->nv, l->nv, &l->M) || coo_to_csr(&rk, l->nv, l->nv, &l->K) ||
        coo_to_csr(&rdx, l->np, l->nv, &l->Dx) || coo_to_csr(&rdy, l->np, l->nv, &l->Dy))
        return -1;
    return 0;
}

/* A = [[M, 0, K, D^T], [0, 0, D, 0], [K, D^T, -alpha^{-1} M, 0], [D, 0, 0, 0]]
 * (eq. (mp3)) with M, K one block per velocity component and D = [D_x, D_y]. */
static int build_A(slevel* l, double alpha) {
    scoo c = {0};
    const scsr* D[2] = {&l->Dx, &l->Dy};
    for (int comp = 0; comp < 2; ++comp) {
        for (int i = 0; i < l->nv; ++i) {
            for (int64_t k = l->M.rowptr[i]; k < l->M.rowptr[i + 1]; ++k) {
                int j = l->M.col[k];
                if (coo_add(&c, off_v(l, comp) + i, off_v(l, comp) + j, l->M.val[k]) ||
                    coo_add(&c, off_l(l, comp) + i, off_l(l, comp) + j, -l->M.val[k] / alpha))
                    return -1;
            }
            for (int64_t k = l->K.rowptr[i]; k < l->K.rowptr[i + 1]; ++k) {
                int j = l->K.col[k];
                if (coo_add(&c, off_v(l, comp) + i, off_l(l, comp) + j, l->K.val[k]) ||
                    coo_add(&c, off_l(l, comp) + i, off_v(l, comp) + j, l->K.val[k]))
                    return -1;
            }
        }
        for (int q = 0; q < l->np; ++q)
            for (int64_t k = D[comp]->rowptr[q]; k < D[comp]->rowptr[q + 1]; ++k) {
                int i = D[comp]->col[k];
                double d = D[comp]->val[k];
                if (coo_add(&c, off_p(l) + q, off_l(l, comp) + i, d) ||   /* D lambda */
                    coo_add(&c, off_mu(l) + q, off_v(l, comp) + i, d) ||  /* D v */
                    coo_add(&c, off_v(l, comp) + i, off_mu(l) + q, d) ||  /* D^T mu */
                    coo_add(&c, off_l(l, comp) + i, off_p(l) + q, d))     /* D^T p */
                    return -1;
            }
    }
    return coo_to_csr(&c, l->m, l->m, &l->A);
}

/* L = blockdiag(W^, P^, alpha^{-1} W^, alpha^{-1} P^),
 * W^ = diag(M + alpha^{1/2} K), P^ = alpha diag(D W^{-1} D^T)  (section 2). */
static void build_L(slevel* l, double alpha) {
    double* W = (double*)malloc((size_t)l->nv * sizeof(double));
    for (int i = 0; i < l->nv; ++i) W[i] = csr_entry(&l->M, i, i) + sqrt(alpha) * csr_entry(&l->K, i, i);
    for (int comp = 0; comp < 2; ++comp)
        for (int i = 0; i < l->nv; ++i) {
            l->Ld[off_v(l, comp) + i] = W[i];
            l->Ld[off_l(l, comp) + i] = W[i] / alpha;
        }
    const scsr* D[2] = {&l->Dx, &l->Dy};
    for (int q = 0; q < l->np; ++q) {
        double s = 0.0;
        for (int comp = 0; comp < 2; ++comp)
            for (int64_t k = D[comp]->rowptr[q]; k < D[comp]->rowptr[q + 1]; ++k)
                s += D[comp]->val[k] * D[comp]->val[k] / W[D[comp]->col[k]];
        l->Ld[off_p(l) + q] = alpha * s;
        l->Ld[off_mu(l) + q] = s;
    }
    free(W);
}

/* N_ii = sum_j A_ji^2 / L_jj (A is symmetric: row i) */
static void build_N(slevel* l) {
    for (int i = 0; i < l->m; ++i) {
        double s = 0.0;
        for (int64_t k = l->A.rowptr[i]; k < l->A.rowptr[i + 1]; ++k) s += l->A.val[k] * l->A.val[k] / l->Ld[l->A.col[k]];
        l->Nd[i] = s;
    }
}

static void build_order(slevel* l, int lexicographic) {
    if (lexicographic) {
        for (int u = 0; u < l->m; ++u) l->order[u] = u;
        return;
    }
    int pos = 0, n = l->n, ng = l->ng;
    for (int blk = 0; blk < 6; ++blk) {
        int vel = blk != 2 && blk != 5;
        int off = blk == 0 ? off_v(l, 0) : blk == 1 ? off_v(l, 1) : blk == 2 ? off_p(l)
                : blk == 3 ? off_l(l, 0) : blk == 4 ? off_l(l, 1) : off_mu(l);
        if (vel) {
            for (int c = 0; c < VCOL; ++c)
                for (int b = 1; b <= ng - 2; ++b)
                    for (int a = 1; a <= ng - 2; ++a)
                        if ((a + 7 * b) % VCOL == c) l->order[pos++] = off + vidx(l, a, b);
        } else {
            for (int c = 0; c < PCOL; ++c)
                for (int j = 0; j <= n; ++j)
                    for (int i = 0; i <= n; ++i)
                        if ((i + 2 * j) % PCOL == c) l->order[pos++] = off + j * (n + 1) + i;
        }
    }
}

/* The canonical embedding of the coarse P2 space into the fine one: each fine
 * interior P2 node takes the value of the coarse function there, evaluated
 * with the coarse P2 basis of the coarse triangle that holds the node. */
static int build_P2(slevel* lf, const slevel* lc) {
    scoo c = {0};
    int ncc = lc->n;
    for (int b = 1; b <= lf->ng - 2; ++b)
        for (int a = 1; a <= lf->ng - 2; ++a) {
            double X = a / 4.0, Y = b / 4.0; /* in coarse cells */
            int I = (int)floor(X), J = (int)floor(Y);
            if (I > ncc - 1) I = ncc - 1;
            if (J > ncc - 1) J = ncc - 1;
            double s = X - I, t = Y - J;
            int vx[3], vy[3];
            double lam[3];
            if (s >= t) { /* lower triangle (I,J), (I+1,J), (I+1,J+1) */
                vx[0] = I; vy[0] = J; vx[1] = I + 1; vy[1] = J; vx[2] = I + 1; vy[2] = J + 1;
                lam[0] = 1.0 - s; lam[1] = s - t; lam[2] = t;
            } else { /* upper triangle (I,J), (I+1,J+1), (I,J+1) */
                vx[0] = I; vy[0] = J; vx[1] = I + 1; vy[1] = J + 1; vx[2] = I; vy[2] = J + 1;
                lam[0] = 1.0 - t; lam[1] = s; lam[2] = t - s;
            }
            int row = vidx(lf, a, b);
            for (int q = 0; q < 6; ++q) {
                double wgt;
                int ca, cb;
                if (q < 3) {
                    wgt = lam[q] * (2.0 * lam[q] - 1.0);
                    ca = 2 * vx[q];
                    cb = 2 * vy[q];
                } else {
                    int u = EDGE[q - 3][0], v = EDGE[q - 3][1];
                    wgt = 4.0 * lam[u] * lam[v];
                    ca = vx[u] + vx[v];
                    cb = vy[u] + vy[v];
                }
                int col = vidx(lc, ca, cb);
                if (wgt != 0.0 && col >= 0 && coo_add(&c, row, col, wgt)) return -1;
            }
        }
    return coo_to_csr(&c, lf->nv, lc->nv, &lf->P2);
}

/* The canonical embedding of the coarse P1 space: linear interpolation on the
 * coarse triangle that holds the fine vertex. */
static int build_P1(slevel* lf, const slevel* lc) {
    scoo c = {0};
    int nf = lf->n, nc = lc->n;
    for (int j = 0; j <= nf; ++j)
        for (int i = 0; i <= nf; ++i) {
            double X = i / 2.0, Y = j / 2.0;
            int I = (int)floor(X), J = (int)floor(Y);
            if (I > nc - 1) I = nc - 1;
            if (J > nc - 1) J = nc - 1;
            double s = X - I, t = Y - J;
            int v[3];
            double lam[3];
            if (s >= t) {
                v[0] = J * (nc + 1) + I; v[1] = J * (nc + 1) + I + 1; v[2] = (J + 1) * (nc + 1) + I + 1;
                lam[0] = 1.0 - s; lam[1] = s - t; lam[2] = t;
            } else {
                v[0] = J * (nc + 1) + I; v[1] = (J + 1) * (nc + 1) + I + 1; v[2] = (J + 1) * (nc + 1) + I;
                lam[0] = 1.0 - t; lam[1] = s; lam[2] = t - s;
            }
            for (int q = 0; q < 3; ++q)
                if (lam[q] != 0.0 && coo_add(&c, j * (nf + 1) + i, v[q], lam[q])) return -1;
        }
    return coo_to_csr(&c, lf->np, lc->np, &lf->P1);
}

/* ------------------------------------------------------- hierarchy --- */

static void level_free(slevel* l) {
    csr_free(&l->Mf); csr_free(&l->Kf); csr_free(&l->Dxf); csr_free(&l->Dyf);
    csr_free(&l->M); csr_free(&l->K); csr_free(&l->Dx); csr_free(&l->Dy);
    csr_free(&l->A); csr_free(&l->P2); csr_free(&l->P1);
    free(l->Ld); free(l->Nd); free(l->w); free(l->order);
    free(l->f); free(l->x); free(l->r); free(l->p);
    memset(l, 0, sizeof(*l));
}

static int lu_factor(int m, double* a, int* piv);

void sto_destroy(shier* H) {
    if (!H) return;
    for (int k = 1; k <= ST_MAXLEV; ++k) level_free(&H->lev[k]);
    free(H->clu);
    free(H->cpiv);
    free(H);
}

shier* sto_create(int L, double alpha, int smoother, int nu_pre, int nu_post, int gamma, double tau,
                  int lexicographic) {
    if (L < 1 || L > ST_MAXLEV || !(alpha > 0.0)) return NULL;
    shier* H = (shier*)calloc(1, sizeof(shier));
    if (!H) return NULL;
    H->L = L;
    H->alpha = alpha;
    H->smoother = smoother;
    H->nu_pre = nu_pre;
    H->nu_post = nu_post;
    H->gamma = gamma;
    H->tau = tau;
    H->lexicographic = lexicographic;
    for (int k = 1; k <= L; ++k) {
        slevel* l = &H->lev[k];
        l->n = 1 << k;
        l->ng = 2 * l->n + 1;
        l->nv = (l->ng - 2) * (l->ng - 2);
        l->np = (l->n + 1) * (l->n + 1);
        l->m = 4 * l->nv + 2 * l->np;
        size_t m = (size_t)l->m;
        if (assemble(l) || build_A(l, alpha)) goto fail;
        l->Ld = (double*)malloc(m * sizeof(double));
        l->Nd = (double*)malloc(m * sizeof(double));
        l->order = (int*)malloc(m * sizeof(int));
        l->f = (double*)calloc(m, sizeof(double));
        l->x = (double*)calloc(m, sizeof(double));
        l->r = (double*)calloc(m, sizeof(double));
        l->p = (double*)calloc(m, sizeof(double));
        if (!l->Ld || !l->Nd || !l->order || !l->f || !l->x || !l->r || !l->p) goto fail;
        build_L(l, alpha);
        build_N(l);
        build_order(l, lexicographic);
        if (k > 1 && (build_P2(l, &H->lev[k - 1]) || build_P1(l, &H->lev[k - 1]))) goto fail;
    }
    {
        /* coarsest level: the bordered system [[S A S, S C], [C^T S, 0]] with
         * S = L^{-1/2} (a symmetric diagonal scaling, which keeps the system
         * well conditioned for every alpha) and C the functionals int p and
         * int mu, dense LU; x = S y */
        slevel* c = &H->lev[1];
        int m = c->m, cm = m + 2;
        H->cm = cm;
        H->clu = (double*)calloc((size_t)cm * cm, sizeof(double));
        H->cpiv = (int*)malloc((size_t)cm * sizeof(int));
        if (!H->clu || !H->cpiv) goto fail;
        for (int i = 0; i < m; ++i)
            for (int64_t k = c->A.rowptr[i]; k < c->A.rowptr[i + 1]; ++k)
                H->clu[(size_t)i * cm + c->A.col[k]] = c->A.val[k] / sqrt(c->Ld[i]) / sqrt(c->Ld[c->A.col[k]]);
        for (int q = 0; q < c->np; ++q) {
            int ip = off_p(c) + q, im = off_mu(c) + q;
            H->clu[(size_t)ip * cm + m] = c->w[q] / sqrt(c->Ld[ip]);
            H->clu[(size_t)m * cm + ip] = c->w[q] / sqrt(c->Ld[ip]);
            H->clu[(size_t)im * cm + m + 1] = c->w[q] / sqrt(c->Ld[im]);
            H->clu[(size_t)(m + 1) * cm + im] = c->w[q] / sqrt(c->Ld[im]);
        }
        if (lu_factor(cm, H->clu, H->cpiv)) goto fail;
    }
    return H;
fail:
    sto_destroy(H);
    return NULL;
}

/* ------------------------------------------------------------ export --- */

static const scsr* pick(const shier* H, int level, int which) {
    const slevel* l = &H->lev[level];
    switch (which) {
    case 0: return &l->M;
    case 1: return &l->K;
    case 2: return &l->Dx;
    case 3: return &l->Dy;
    case 4: return &l->A;
    case 5: return &l->P2;
    case 6: return &l->P1;
    case 7: return &l->Mf;
    case 8: return &l->Kf;
    case 9: return &l->Dxf;
    default: return &l->Dyf;
    }
}

void sto_sizes(const shier* H, int level, int* out) {
    const slevel* l = &H->lev[level];
    out[0] = l->n;
    out[1] = l->nv;
    out[2] = l->np;
    out[3] = l->m;
}
int64_t sto_csr_nnz(const shier* H, int level, int which) { return pick(H, level, which)->nnz; }
void sto_csr_shape(const shier* H, int level, int which, int* shape) {
    shape[0] = pick(H, level, which)->nrows;
    shape[1] = pick(H, level, which)->ncols;
}
void sto_csr_export(const shier* H, int level, int which, int64_t* rowptr, int* col, double* val) {
    const scsr* m = pick(H, level, which);
    memcpy(rowptr, m->rowptr, ((size_t)m->nrows + 1) * sizeof(int64_t));
    memcpy(col, m->col, (size_t)m->nnz * sizeof(int));
    memcpy(val, m->val, (size_t)m->nnz * sizeof(double));
}
void sto_ldiag(const shier* H, int level, double* out) { memcpy(out, H->lev[level].Ld, (size_t)H->lev[level].m * sizeof(double)); }
void sto_ndiag(const shier* H, int level, double* out) { memcpy(out, H->lev[level].Nd, (size_t)H->lev[level].m * sizeof(double)); }
void sto_order(const shier* H, int level, int* out) { memcpy(out, H->lev[level].order, (size_t)H->lev[level].m * sizeof(int)); }
void sto_pweights(const shier* H, int level, double* out) { memcpy(out, H->lev[level].w, (size_t)H->lev[level].np * sizeof(double)); }

/* ------------------------------------------------------- basic ops --- */

/* f = (M v_D, 0, 0, 0): v_D given per component at all ng^2 P2 nodes
 * (component-major), weighted by the full P2 mass matrix */
void sto_rhs(const shier* H, const double* vD, double* f) {
    const slevel* l = &H->lev[H->L];
    int ng2 = l->ng * l->ng;
    for (int i = 0; i < l->m; ++i) f[i] = 0.0;
    for (int comp = 0; comp < 2; ++comp)
        for (int gi = 0; gi < ng2; ++gi) {
            int vi = vidx(l, gi % l->ng, gi / l->ng);
            if (vi < 0) continue;
            double s = 0.0;
            for (int64_t k = l->Mf.rowptr[gi]; k < l->Mf.rowptr[gi + 1]; ++k) s += l->Mf.val[k] * vD[comp * ng2 + l->Mf.col[k]];
            f[off_v(l, comp) + vi] = s;
        }
}

void sto_residual(const shier* H, int level, const double* f, const double* x, double* r) {
    const slevel* l = &H->lev[level];
    csr_mv(&l->A, x, r);
    for (int i = 0; i < l->m; ++i) r[i] = f[i] - r[i];
}

/* remove the means of p and mu (int p = int mu = 0; sum_q w_q = |Omega| = 1) */
void sto_normalize(const shier* H, int level, double* x) {
    const slevel* l = &H->lev[level];
    double sp = 0.0, sm = 0.0, sw = 0.0;
    for (int q = 0; q < l->np; ++q) {
        sp += l->w[q] * x[off_p(l) + q];
        sm += l->w[q] * x[off_mu(l) + q];
        sw += l->w[q];
    }
    for (int q = 0; q < l->np; ++q) {
        x[off_p(l) + q] -= sp / sw;
        x[off_mu(l) + q] -= sm / sw;
    }
}

double sto_norm_Linv(const shier* H, int level, const double* v) {
    const slevel* l = &H->lev[level];
    double s = 0.0;
    for (int i = 0; i < l->m; ++i) s += v[i] * v[i] / l->Ld[i];
    return sqrt(s);
}

double sto_norm_L(const shier* H, int level, const double* v) {
    const slevel* l = &H->lev[level];
    double s = 0.0;
    for (int i = 0; i < l->m; ++i) s += v[i] * v[i] * l->Ld[i];
    return sqrt(s);
}

/* --------------------------------------------------------- smoothers --- */
/* A is symmetric, so the column A_{:,i} of Algorithms 1 and 2 is row i. */

/* Algorithm 1: x <- x + tau L^{-1} A^T L^{-1} r, r updated alongside */
static void ne_step(slevel* l, double tau, double* x, double* r) {
    const scsr* A = &l->A;
    for (int i = 0; i < l->m; ++i) {
        double q = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) q += A->val[k] / l->Ld[A->col[k]] * r[A->col[k]];
        l->p[i] = tau * q / l->Ld[i];
    }
    for (int i = 0; i < l->m; ++i) {
        x[i] += l->p[i];
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) r[A->col[k]] -= A->val[k] * l->p[i];
    }
}

/* Algorithm 2: Gauss-Seidel on N = A^T L^{-1} A in the order `order`
 * (reversed for the second half of an sLSGS step) */
static void lsgs_step(slevel* l, int reverse, double* x, double* r) {
    const scsr* A = &l->A;
    for (int s = 0; s < l->m; ++s) {
        int i = l->order[reverse ? l->m - 1 - s : s];
        double q = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) q += A->val[k] / l->Ld[A->col[k]] * r[A->col[k]];
        double p = q / l->Nd[i];
        x[i] += p;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) r[A->col[k]] -= A->val[k] * p;
    }
}

void sto_smooth(shier* H, int level, const double* f, double* x, int steps) {
    slevel* l = &H->lev[level];
    sto_residual(H, level, f, x, l->r);
    for (int m = 0; m < steps; ++m) {
        if (H->smoother == 0) {
            ne_step(l, H->tau, x, l->r);
        } else {
            lsgs_step(l, 0, x, l->r);
            if (H->smoother == 2) lsgs_step(l, 1, x, l->r);
        }
    }
}

/* ------------------------------------------------------- transfers --- */

static void restrict_block(const scsr* P, const double* rf, double* rc) {
    for (int i = 0; i < P->ncols; ++i) rc[i] = 0.0;
    for (int i = 0; i < P->nrows; ++i)
        for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) rc[P->col[k]] += P->val[k] * rf[i];
}

static void prolong_block(const scsr* P, const double* xc, double* xf) {
    for (int i = 0; i < P->nrows; ++i) {
        double s = 0.0;
        for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) s += P->val[k] * xc[P->col[k]];
        xf[i] += s;
    }
}

/* rc = I^T rf block by block (P2 embedding for v and lambda, P1 for p and mu) */
void sto_restrict(const shier* H, int level, const double* rf, double* rc) {
    const slevel* f = &H->lev[level];
    const slevel* c = &H->lev[level - 1];
    for (int comp = 0; comp < 2; ++comp) {
        restrict_block(&f->P2, rf + off_v(f, comp), rc + off_v(c, comp));
        restrict_block(&f->P2, rf + off_l(f, comp), rc + off_l(c, comp));
    }
    restrict_block(&f->P1, rf + off_p(f), rc + off_p(c));
    restrict_block(&f->P1, rf + off_mu(f), rc + off_mu(c));
}

void sto_prolong_add(const shier* H, int level, const double* xc, double* xf) {
    const slevel* f = &H->lev[level];
    const slevel* c = &H->lev[level - 1];
    for (int comp = 0; comp < 2; ++comp) {
        prolong_block(&f->P2, xc + off_v(c, comp), xf + off_v(f, comp));
        prolong_block(&f->P2, xc + off_l(c, comp), xf + off_l(f, comp));
    }
    prolong_block(&f->P1, xc + off_p(c), xf + off_p(f));
    prolong_block(&f->P1, xc + off_mu(c), xf + off_mu(f));
}

/* ------------------------------------------------------- coarse solve --- */

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

/* exact solve on the coarsest grid (h = 1/2): the solution of A x = f with
 * int p = int mu = 0 (f must be orthogonal to the kernel, which every
 * restricted residual is) */
void sto_coarse_solve(const shier* H, const double* f, double* x) {
    const slevel* c = &H->lev[1];
    int m = c->m;
    double* b = (double*)malloc((size_t)H->cm * sizeof(double));
    for (int i = 0; i < m; ++i) b[i] = f[i] / sqrt(c->Ld[i]);
    b[m] = b[m + 1] = 0.0;
    lu_solve(H->cm, H->clu, H->cpiv, b);
    for (int i = 0; i < m; ++i) x[i] = b[i] / sqrt(c->Ld[i]);
    free(b);
}

/* ------------------------------------------------------- multigrid --- */

static void cycle_rec(shier* H, int k, const double* f, double* x) {
    if (k == 1) {
        sto_coarse_solve(H, f, x);
        return;
    }
    slevel* l = &H->lev[k];
    slevel* c = &H->lev[k - 1];
    if (H->nu_pre > 0) sto_smooth(H, k, f, x, H->nu_pre);
    sto_residual(H, k, f, x, l->r);
    sto_restrict(H, k, l->r, c->f);
    for (int i = 0; i < c->m; ++i) c->x[i] = 0.0;
    for (int g = 0; g < H->gamma; ++g) cycle_rec(H, k - 1, c->f, c->x);
    sto_prolong_add(H, k, c->x, x);
    if (H->nu_post > 0) sto_smooth(H, k, f, x, H->nu_post);
}

void sto_cycle(shier* H, int level, const double* f, double* x) { cycle_rec(H, level, f, x); }

/* cycles until ||f - A x||_{L^{-1}} <= tol ||f||_{L^{-1}} or max_iter */
int sto_solve(shier* H, const double* f, double* x, double tol, int max_iter, double* relres, double* history) {
    int L = H->L;
    slevel* l = &H->lev[L];
    double fn = sto_norm_Linv(H, L, f);
    if (fn == 0.0) fn = 1.0;
    int it = 0;
    double rr;
    for (;;) {
        sto_residual(H, L, f, x, l->r);
        rr = sto_norm_Linv(H, L, l->r) / fn;
        if (history) history[it] = rr;
        if (rr <= tol || it >= max_iter || !(rr == rr)) break;
        cycle_rec(H, L, f, x);
        ++it;
    }
    if (relres) *relres = rr;
    return it;
}

/* Section 3 protocol: zero right-hand side, initial guess x0, iterate until the
 * error (x0 with the means of p and mu removed; the solution is 0) has dropped
 * by `reduction` in ||.||_L.  Returns the iterations, -1 beyond max_iter. */
int sto_protocol_iterations(shier* H, double* x0, double reduction, int max_iter) {
    int L = H->L;
    slevel* l = &H->lev[L];
    double* zero = (double*)calloc((size_t)l->m, sizeof(double));
    double* e = (double*)malloc((size_t)l->m * sizeof(double));
    if (!zero || !e) {
        free(zero);
        free(e);
        return -2;
    }
    memcpy(e, x0, (size_t)l->m * sizeof(double));
    sto_normalize(H, L, e);
    double e0 = sto_norm_L(H, L, e);
    int it = 0;
    for (;;) {
        memcpy(e, x0, (size_t)l->m * sizeof(double));
        sto_normalize(H, L, e);
        if (sto_norm_L(H, L, e) <= reduction * e0) break;
        if (it >= max_iter) {
            it = -1;
            break;
        }
        cycle_rec(H, L, zero, x0);
        ++it;
    }
    free(zero);
    free(e);
    return it;
}
