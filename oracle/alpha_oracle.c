/*
 * Exact CPU oracle for the alpha complex of a set of weighted points
 * (Masood, Ray, Natarajan, "Parallel Computation of Alpha Complexes for
 * Biomolecules", arXiv 1908.05944).
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, exact reference that the
 * CUDA library is checked against. Only the tests, the smoke check and the
 * bench's CPU-baseline leg load it; the library never calls it, and the two
 * share no source.
 *
 * What it computes, in the paper's order:
 *   quantise: X = round_half_even(1024 x), R = round_half_even(1024 r),
 *             W = R^2, A = round_half_even(2^20 alpha)   (1/1024 A units)
 *   Step 1 (Section 3.1): Sigma_ortho^d = { sigma : OrthoSize(sigma) <= alpha },
 *             built bottom-up over edges, triangles, tetrahedra because the
 *             OrthoSize of a face never exceeds that of the simplex (Section 4.3)
 *   Step 2:   K^3 = tetrahedra of Sigma_ortho^3 that satisfy AC2 at their
 *             orthocentre (Definition "Alpha complex", AC1-AC3, Section 2.4)
 *   Step 3:   K^2 = Facets(K^3) + free triangles that satisfy AC2
 *   Step 4:   K^1 = Facets(K^2) + free edges that satisfy AC2
 *   Step 5:   K^0 = endpoints of K^1 + free vertices whose centre satisfies AC2
 *   filtration value: Size (Section 2.3) = OrthoSize when AC2 holds at the
 *             orthocentre ("unattached"), else the smallest Size of a coface
 *             one dimension up that lies in the complex (the closest witness of
 *             an attached simplex is a witness of a coface with the same Size,
 *             as in the proofs of Lemmas 1 and 2).
 *
 * Geometry, in exact integers. For sigma = (v0..vd), q_k = P_vk - P_v0 and
 * a_k = |q_k|^2 - W_vk + W_v0 (k = 1..d). A point p = P_v0 + y has equal power
 * to all vertices (AC1) iff 2 q_k . y = a_k for all k. The orthocentre is the
 * minimum-norm such y: y = sum_k mu_k q_k with G mu = a / 2, G the Gram matrix
 * of the q_k. With adj(G) the adjugate and g = det G > 0:
 *   n = adj(G) a,  y = (sum_k n_k q_k) / (2g),
 *   OrthoSize = |y|^2 - W_v0 = (n . a - 4 g W_v0) / (4 g).
 * For a test ball x, Delta_x = pi(c, b_x) - pi(c, b_v0) = a_x - 2 q_x . y with
 * a_x = |q_x|^2 - W_x + W_v0; AC2 fails at c iff some x has Delta_x < 0.
 *
 * Ties (degeneracies, Section 2: "symbolic perturbation"): the weights are
 * perturbed W_k -> W_k + eps_k with eps_k decreasing steeply in the input index
 * k. Delta_x is affine in the weights: its coefficient on W_x is -1, on W_vk
 * (k >= 1) it is beta_k, and on W_v0 it is 1 - sum beta, where beta =
 * G^-1 (q_1.q_x, .., q_d.q_x) are the affine coordinates of the projection of
 * P_x on the affine hull of sigma. If Delta_x = 0 its perturbed sign is the
 * sign of the coefficient of the smallest input index among sigma and x whose
 * coefficient is non-zero. The AC3 test (OrthoSize <= alpha) is not perturbed.
 * Collinear triples and coplanar quadruples (g = 0) have no orthocentre and are
 * never simplices.
 *
 * Candidate sets (why the search is complete): a simplex in Sigma_ortho has
 * OrthoSize <= A, so its orthocentre c lies within sqrt(W_v + A) <= h of every
 * vertex v (h^2 = max W + A). A ball x that violates AC2 at c, ties included,
 * has pi(c, b_x) <= A, so |c - P_x| <= h and |P_x - P_v0| <= 2h. An edge in
 * Sigma_ortho^1 joins balls whose grown spheres meet, so its length is <= 2h.
 * The oracle therefore looks only at atoms within 2h of P_v0 (all atoms when
 * alpha is infinite).
 *
 * Integer ranges: every coordinate difference that enters a product is checked
 * to be at most 2^14 quanta (16 A) per axis and W + |A| <= 2^26; under these
 * bounds every quantity above fits in a signed 128-bit integer. Outside them
 * the oracle returns an error instead of overflowing.
 *
 * Filtration values are returned in A^2 as num / (den * 2^20), evaluated in
 * long double and rounded to double (within one ulp of the exact rational).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_DEGENERATE -2
#define OR_ERR_RANGE -3
#define OR_ERR_OOM -5

#define COORD_LIMIT (1LL << 14)
#define WEIGHT_LIMIT (1LL << 26)

/* ------------------------------------------------------------------ */
/* growable arrays                                                     */

typedef struct {
    int32_t *v;
    int64_t n, cap;
} ivec;

static int iv_push(ivec *a, int32_t x) {
    if (a->n == a->cap) {
        int64_t c = a->cap ? 2 * a->cap : 64;
        int32_t *p = (int32_t *)realloc(a->v, (size_t)c * sizeof(int32_t));
        if (!p) return -1;
        a->v = p;
        a->cap = c;
    }
    a->v[a->n++] = x;
    return 0;
}

static void iv_free(ivec *a) {
    free(a->v);
    a->v = NULL;
    a->n = a->cap = 0;
}

/* ------------------------------------------------------------------ */
/* problem                                                             */

typedef struct {
    int64_t n;
    int64_t *P; /* 3n quantised centres */
    int64_t *W; /* n squared quantised radii */
    int64_t A;
    int inf;     /* alpha = +infinity: no AC3 test, every atom a candidate */
    int64_t H2;  /* max W + A */
    int64_t *nb_off;
    int32_t *nb; /* per atom: atoms within 2h, ascending input index */
    int nthreads;
    volatile int range_error;
} problem;

/* Simplex lists: flat arrays of (d+1) ascending input indices, sorted lexicographically. */
typedef struct {
    int32_t *v;
    int64_t n;
} slist;

typedef struct oracle_result {
    int64_t n_atoms;
    slist sigma[4];    /* Sigma_ortho^d */
    slist K[4];        /* alpha complex by dimension */
    uint8_t *attached[4];
    double *f[4];      /* filtration value (Size) in A^2 */
    double *orthosize[4];
    int32_t *src_dim[4];
    int64_t *src_idx[4];
    problem *prob;
} oracle_result;

/* ------------------------------------------------------------------ */
/* geometry of one simplex                                             */

typedef struct {
    int d;
    int64_t q[3][3];
    int64_t a[3];
    i128 g;         /* det G */
    i128 adj[3][3]; /* adjugate of G */
    i128 nv[3];     /* adj(G) a */
    i128 ynum[3];   /* sum_k nv_k q_k ; y = ynum / (2g) */
    i128 os_num;    /* OrthoSize = os_num / os_den */
    i128 os_den;
} geom;

static int check_diff(problem *pr, int64_t dx, int64_t dy, int64_t dz) {
    if (dx > COORD_LIMIT || dx < -COORD_LIMIT || dy > COORD_LIMIT || dy < -COORD_LIMIT || dz > COORD_LIMIT ||
        dz < -COORD_LIMIT) {
        pr->range_error = 1;
        return 0;
    }
    return 1;
}

/* Returns 1 if the simplex is non-degenerate (det G > 0), else 0. */
static int simplex_geom(problem *pr, const int32_t *v, int d, geom *s) {
    s->d = d;
    const int64_t *P = pr->P, *W = pr->W;
    int64_t w0 = W[v[0]];
    if (d == 0) {
        s->g = 1;
        s->os_num = -(i128)w0;
        s->os_den = 1;
        return 1;
    }
    for (int k = 0; k < d; k++) {
        for (int c = 0; c < 3; c++) s->q[k][c] = P[3 * v[k + 1] + c] - P[3 * v[0] + c];
        if (!check_diff(pr, s->q[k][0], s->q[k][1], s->q[k][2])) return 0;
        s->a[k] = s->q[k][0] * s->q[k][0] + s->q[k][1] * s->q[k][1] + s->q[k][2] * s->q[k][2] - W[v[k + 1]] + w0;
    }
    i128 G[3][3];
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++)
            G[i][j] = (i128)s->q[i][0] * s->q[j][0] + (i128)s->q[i][1] * s->q[j][1] + (i128)s->q[i][2] * s->q[j][2];
    if (d == 1) {
        s->g = G[0][0];
        s->adj[0][0] = 1;
    } else if (d == 2) {
        s->g = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        s->adj[0][0] = G[1][1];
        s->adj[0][1] = -G[0][1];
        s->adj[1][0] = -G[1][0];
        s->adj[1][1] = G[0][0];
    } else {
        /* cofactor C_ij = (-1)^(i+j) M_ij; adj = C^T (G symmetric, so adj is symmetric) */
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
                /* cyclic index choice makes the sign come out right */
                s->adj[j][i] = G[r0][c0] * G[r1][c1] - G[r0][c1] * G[r1][c0];
            }
        s->g = G[0][0] * s->adj[0][0] + G[0][1] * s->adj[1][0] + G[0][2] * s->adj[2][0];
    }
    if (s->g <= 0) return 0; /* Gram determinant is >= 0; zero means a flat simplex */
    i128 na = 0;
    for (int i = 0; i < d; i++) {
        s->nv[i] = 0;
        for (int j = 0; j < d; j++) s->nv[i] += s->adj[i][j] * s->a[j];
        na += s->nv[i] * s->a[i];
    }
    for (int c = 0; c < 3; c++) {
        s->ynum[c] = 0;
        for (int k = 0; k < d; k++) s->ynum[c] += s->nv[k] * s->q[k][c];
    }
    s->os_num = na - 4 * s->g * (i128)w0;
    s->os_den = 4 * s->g;
    return 1;
}

/* AC3: OrthoSize(sigma) <= alpha (inclusive, unperturbed). */
static int ac3_holds(problem *pr, const geom *s) {
    if (pr->inf) return 1;
    return s->os_num <= (i128)pr->A * s->os_den;
}

/* Sign of Delta_x under the symbolic perturbation of the weights (+1 or -1). */
static int sos_sign(const int32_t *v, const geom *s, int32_t x, const int64_t qx[3]) {
    int d = s->d;
    i128 coef[4];
    int32_t who[4];
    if (d == 0) {
        coef[0] = 1;
    } else {
        i128 gx[3], proj[3], sum = 0;
        for (int k = 0; k < d; k++) gx[k] = (i128)s->q[k][0] * qx[0] + (i128)s->q[k][1] * qx[1] + (i128)s->q[k][2] * qx[2];
        for (int k = 0; k < d; k++) {
            proj[k] = 0;
            for (int j = 0; j < d; j++) proj[k] += s->adj[k][j] * gx[j];
            sum += proj[k];
        }
        coef[0] = s->g - sum; /* g * (1 - sum beta) */
        for (int k = 0; k < d; k++) coef[k + 1] = proj[k]; /* g * beta_k */
    }
    for (int k = 0; k <= d; k++) who[k] = v[k];
    /* smallest input index with a non-zero coefficient decides; x's own coefficient is -1 */
    int32_t best = x;
    int sign = -1;
    for (int k = 0; k <= d; k++) {
        if (coef[k] != 0 && who[k] < best) {
            best = who[k];
            sign = coef[k] > 0 ? 1 : -1;
        }
    }
    return sign;
}

/* Does ball x violate AC2 at the orthocentre of sigma (perturbed sense)? */
static int violates(problem *pr, const int32_t *v, const geom *s, int32_t x) {
    const int64_t *P = pr->P, *W = pr->W;
    int64_t qx[3];
    for (int c = 0; c < 3; c++) qx[c] = P[3 * x + c] - P[3 * v[0] + c];
    if (!check_diff(pr, qx[0], qx[1], qx[2])) return 0;
    int64_t ax = qx[0] * qx[0] + qx[1] * qx[1] + qx[2] * qx[2] - W[x] + W[v[0]];
    i128 val;
    if (s->d == 0) {
        val = ax;
    } else {
        /* (Delta_x) * g = a_x g - q_x . ynum ; g > 0 */
        val = (i128)ax * s->g - ((i128)qx[0] * s->ynum[0] + (i128)qx[1] * s->ynum[1] + (i128)qx[2] * s->ynum[2]);
    }
    if (val < 0) return 1;
    if (val > 0) return 0;
    return sos_sign(v, s, x, qx) < 0;
}

/* AC2 at the orthocentre of sigma (at P_v0 for a vertex). */
static int ac2_holds(problem *pr, const int32_t *v, int d, const geom *s) {
    int64_t lo = pr->inf ? 0 : pr->nb_off[v[0]], hi = pr->inf ? pr->n : pr->nb_off[v[0] + 1];
    for (int64_t t = lo; t < hi; t++) {
        int32_t x = pr->inf ? (int32_t)t : pr->nb[t];
        int in = 0;
        for (int k = 0; k <= d; k++) in |= (v[k] == x);
        if (in) continue;
        if (violates(pr, v, s, x)) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* parallel loop over owner atoms, results concatenated in owner order */

typedef struct {
    problem *pr;
    int64_t n_items;
    int64_t chunk;
    int64_t n_chunks;
    int64_t next;
    pthread_mutex_t mu;
    void *ctx;
    int (*body)(problem *, void *, int64_t item, ivec *out);
    ivec *outs; /* one per chunk */
    int err;
} pfor;

static void *pfor_worker(void *arg) {
    pfor *p = (pfor *)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        int64_t c = p->next++;
        pthread_mutex_unlock(&p->mu);
        if (c >= p->n_chunks) break;
        int64_t lo = c * p->chunk, hi = lo + p->chunk < p->n_items ? lo + p->chunk : p->n_items;
        for (int64_t i = lo; i < hi; i++)
            if (p->body(p->pr, p->ctx, i, &p->outs[c])) {
                p->err = OR_ERR_OOM;
                return NULL;
            }
    }
    return NULL;
}

/* Runs body over [0, n_items); concatenates outputs in item order into *out. */
static int parallel_collect(problem *pr, int64_t n_items, void *ctx,
                            int (*body)(problem *, void *, int64_t, ivec *), ivec *out) {
    pfor p;
    memset(&p, 0, sizeof(p));
    p.pr = pr;
    p.n_items = n_items;
    p.chunk = 64;
    p.n_chunks = (n_items + p.chunk - 1) / p.chunk;
    p.ctx = ctx;
    p.body = body;
    p.outs = (ivec *)calloc((size_t)(p.n_chunks ? p.n_chunks : 1), sizeof(ivec));
    if (!p.outs) return OR_ERR_OOM;
    pthread_mutex_init(&p.mu, NULL);
    int nt = pr->nthreads > 0 ? pr->nthreads : 1;
    pthread_t th[256];
    if (nt > 256) nt = 256;
    for (int t = 0; t < nt; t++) pthread_create(&th[t], NULL, pfor_worker, &p);
    for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&p.mu);
    int64_t total = 0;
    for (int64_t c = 0; c < p.n_chunks; c++) total += p.outs[c].n;
    out->v = (int32_t *)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
    out->n = 0;
    out->cap = total;
    if (!out->v) p.err = OR_ERR_OOM;
    for (int64_t c = 0; c < p.n_chunks; c++) {
        if (out->v && p.outs[c].n) memcpy(out->v + out->n, p.outs[c].v, (size_t)p.outs[c].n * sizeof(int32_t));
        out->n += p.outs[c].n;
        iv_free(&p.outs[c]);
    }
    free(p.outs);
    return p.err;
}

/* ------------------------------------------------------------------ */
/* lexicographic search in a sorted simplex list                        */

static int cmp_tuple(const int32_t *a, const int32_t *b, int k) {
    for (int i = 0; i < k; i++) {
        if (a[i] < b[i]) return -1;
        if (a[i] > b[i]) return 1;
    }
    return 0;
}

static int64_t find_tuple(const slist *L, int d, const int32_t *t) {
    int64_t lo = 0, hi = L->n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp_tuple(L->v + mid * (d + 1), t, d + 1);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

/* one comparator per tuple width (no shared state: concurrent oracle runs
   on several host threads each sort their own lists) */
static int qsort_cmp1(const void *a, const void *b) { return cmp_tuple((const int32_t *)a, (const int32_t *)b, 1); }
static int qsort_cmp2(const void *a, const void *b) { return cmp_tuple((const int32_t *)a, (const int32_t *)b, 2); }
static int qsort_cmp3(const void *a, const void *b) { return cmp_tuple((const int32_t *)a, (const int32_t *)b, 3); }
static int qsort_cmp4(const void *a, const void *b) { return cmp_tuple((const int32_t *)a, (const int32_t *)b, 4); }

/* sort + unique in place; tuples have k (1..4) entries */
static int64_t sort_unique(int32_t *v, int64_t n, int k) {
    if (n == 0) return 0;
    int (*cmp)(const void *, const void *) = k == 1 ? qsort_cmp1 : k == 2 ? qsort_cmp2 : k == 3 ? qsort_cmp3 : qsort_cmp4;
    qsort(v, (size_t)n, (size_t)k * sizeof(int32_t), cmp);
    int64_t m = 1;
    for (int64_t i = 1; i < n; i++)
        if (cmp_tuple(v + (i - 1) * k, v + i * k, k) != 0) {
            if (m != i) memmove(v + m * k, v + i * k, (size_t)k * sizeof(int32_t));
            m++;
        }
    return m;
}

/* ------------------------------------------------------------------ */
/* Step 1: Sigma_ortho, bottom-up                                       */

typedef struct {
    int64_t *up_off; /* Sigma^1 as upper adjacency: j > i */
    int32_t *up;
    slist *s2;
} s1ctx;

static int body_sigma1(problem *pr, void *ctx, int64_t i, ivec *out) {
    (void)ctx;
    int32_t v[2];
    v[0] = (int32_t)i;
    int64_t lo = pr->inf ? 0 : pr->nb_off[i], hi = pr->inf ? pr->n : pr->nb_off[i + 1];
    for (int64_t t = lo; t < hi; t++) {
        int32_t j = pr->inf ? (int32_t)t : pr->nb[t];
        if (j <= i) continue;
        v[1] = j;
        geom s;
        if (!simplex_geom(pr, v, 1, &s)) continue;
        if (!ac3_holds(pr, &s)) continue;
        if (iv_push(out, (int32_t)i) || iv_push(out, j)) return -1;
    }
    return 0;
}

static int in_sorted(const int32_t *a, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        int64_t m = (lo + hi) / 2;
        if (a[m] == x) return 1;
        if (a[m] < x) lo = m + 1;
        else hi = m;
    }
    return 0;
}

static int body_sigma2(problem *pr, void *ctx, int64_t i, ivec *out) {
    s1ctx *c = (s1ctx *)ctx;
    for (int64_t a = c->up_off[i]; a < c->up_off[i + 1]; a++) {
        int32_t j = c->up[a];
        for (int64_t b = a + 1; b < c->up_off[i + 1]; b++) {
            int32_t k = c->up[b];
            if (!in_sorted(c->up, c->up_off[j], c->up_off[j + 1], k)) continue;
            int32_t v[3] = {(int32_t)i, j, k};
            geom s;
            if (!simplex_geom(pr, v, 2, &s)) continue;
            if (!ac3_holds(pr, &s)) continue;
            if (iv_push(out, v[0]) || iv_push(out, v[1]) || iv_push(out, v[2])) return -1;
        }
    }
    return 0;
}

static int body_sigma3(problem *pr, void *ctx, int64_t t, ivec *out) {
    s1ctx *c = (s1ctx *)ctx;
    const int32_t *tri = c->s2->v + 3 * t;
    int32_t i = tri[0], j = tri[1], k = tri[2];
    for (int64_t b = c->up_off[k]; b < c->up_off[k + 1]; b++) {
        int32_t l = c->up[b];
        int32_t f1[3] = {i, j, l}, f2[3] = {i, k, l}, f3[3] = {j, k, l};
        if (find_tuple(c->s2, 2, f1) < 0 || find_tuple(c->s2, 2, f2) < 0 || find_tuple(c->s2, 2, f3) < 0) continue;
        int32_t v[4] = {i, j, k, l};
        geom s;
        if (!simplex_geom(pr, v, 3, &s)) continue;
        if (!ac3_holds(pr, &s)) continue;
        if (iv_push(out, i) || iv_push(out, j) || iv_push(out, k) || iv_push(out, l)) return -1;
    }
    return 0;
}

/* AC2 flags of a simplex list, in parallel */
typedef struct {
    const slist *L;
    int d;
} ac2ctx;

static int body_ac2(problem *pr, void *ctx, int64_t t, ivec *out) {
    ac2ctx *c = (ac2ctx *)ctx;
    const int32_t *v = c->L->v + (c->d + 1) * t;
    geom s;
    int ok = simplex_geom(pr, v, c->d, &s) && ac2_holds(pr, v, c->d, &s);
    return iv_push(out, ok);
}

static int ac2_flags(problem *pr, const slist *L, int d, ivec *flags) {
    ac2ctx c = {L, d};
    return parallel_collect(pr, L->n, &c, body_ac2, flags);
}

/* ------------------------------------------------------------------ */
/* grid of cells of side >= 2h, for the neighbour lists                 */

typedef struct {
    int64_t key;
    int32_t atom;
} keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->atom < y->atom ? -1 : (x->atom > y->atom);
}

static int64_t cell_of(int64_t X, int64_t side) { return (int64_t)floorl((long double)X / (long double)side); }

static int64_t pack_cell(int64_t cx, int64_t cy, int64_t cz) {
    return ((cx + (1LL << 20)) << 42) | ((cy + (1LL << 20)) << 21) | (cz + (1LL << 20));
}

static int64_t find_cell(const keyed *k, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t m = (lo + hi) / 2;
        if (k[m].key < key) lo = m + 1;
        else hi = m;
    }
    return lo;
}

typedef struct {
    keyed *cells;
    int64_t side;
    int64_t limit; /* squared distance bound 4 H2 */
} nbctx;

static int body_nb(problem *pr, void *ctx, int64_t i, ivec *out) {
    nbctx *c = (nbctx *)ctx;
    const int64_t *P = pr->P;
    int64_t cx = cell_of(P[3 * i], c->side), cy = cell_of(P[3 * i + 1], c->side), cz = cell_of(P[3 * i + 2], c->side);
    ivec tmp = {0};
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int64_t key = pack_cell(cx + dx, cy + dy, cz + dz);
                for (int64_t s = find_cell(c->cells, pr->n, key); s < pr->n && c->cells[s].key == key; s++) {
                    int32_t x = c->cells[s].atom;
                    if (x == i) continue;
                    int64_t ex = P[3 * x] - P[3 * i], ey = P[3 * x + 1] - P[3 * i + 1], ez = P[3 * x + 2] - P[3 * i + 2];
                    int64_t d2 = ex * ex + ey * ey + ez * ez;
                    if (d2 == 0) pr->range_error = 2; /* coincident centres */
                    if (d2 <= c->limit && iv_push(&tmp, x)) return -1;
                }
            }
    /* ascending input index */
    if (tmp.n) qsort(tmp.v, (size_t)tmp.n, sizeof(int32_t), cmp_i32);
    if (iv_push(out, (int32_t)tmp.n)) return -1;
    for (int64_t t = 0; t < tmp.n; t++)
        if (iv_push(out, tmp.v[t])) return -1;
    iv_free(&tmp);
    return 0;
}

static int build_neighbours(problem *pr) {
    int64_t n = pr->n;
    pr->nb_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!pr->nb_off) return OR_ERR_OOM;
    if (pr->inf) {
        /* every atom is a candidate; still reject coincident centres */
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = i + 1; j < n; j++)
                if (pr->P[3 * i] == pr->P[3 * j] && pr->P[3 * i + 1] == pr->P[3 * j + 1] &&
                    pr->P[3 * i + 2] == pr->P[3 * j + 2])
                    return OR_ERR_DEGENERATE;
        return OR_OK;
    }
    /* cell side: smallest integer s with s^2 >= 4 H2, so pairs within 2h are in adjacent cells */
    int64_t limit = 4 * pr->H2;
    int64_t side = (int64_t)sqrtl((long double)limit);
    while (side * side < limit) side++;
    if (side < 1) side = 1;
    keyed *cells = (keyed *)malloc((size_t)(n ? n : 1) * sizeof(keyed));
    if (!cells) return OR_ERR_OOM;
    for (int64_t i = 0; i < n; i++) {
        cells[i].key = pack_cell(cell_of(pr->P[3 * i], side), cell_of(pr->P[3 * i + 1], side),
                                 cell_of(pr->P[3 * i + 2], side));
        cells[i].atom = (int32_t)i;
    }
    qsort(cells, (size_t)n, sizeof(keyed), cmp_keyed);
    nbctx c = {cells, side, limit};
    ivec packed = {0};
    int rc = parallel_collect(pr, n, &c, body_nb, &packed);
    free(cells);
    if (rc) return rc;
    if (pr->range_error == 2) {
        iv_free(&packed);
        return OR_ERR_DEGENERATE;
    }
    /* unpack [count, ids...] records */
    int64_t total = packed.n - n;
    pr->nb = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!pr->nb) return OR_ERR_OOM;
    int64_t p = 0, w = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t cnt = packed.v[p++];
        pr->nb_off[i] = w;
        for (int32_t t = 0; t < cnt; t++) pr->nb[w++] = packed.v[p++];
    }
    pr->nb_off[n] = w;
    iv_free(&packed);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Steps 2-5                                                            */

static slist take(ivec *a, int k) {
    slist s;
    s.v = a->v;
    s.n = a->n / k;
    a->v = NULL;
    a->n = a->cap = 0;
    return s;
}

/* Facets of every simplex of L (dimension d), sorted and unique. */
static slist facets_of(const slist *L, int d) {
    ivec out = {0};
    for (int64_t t = 0; t < L->n; t++) {
        const int32_t *v = L->v + (d + 1) * t;
        for (int drop = 0; drop <= d; drop++)
            for (int k = 0; k <= d; k++)
                if (k != drop) iv_push(&out, v[k]);
    }
    slist F;
    F.v = out.v;
    F.n = sort_unique(out.v, out.n / d, d);
    return F;
}

/* K^d = F^d union { sigma in Sigma^d \ F^d : AC2 } (Steps 3-5). */
static int step_lower(problem *pr, const slist *sigma, const slist *F, int d, slist *K) {
    /* free simplices: Sigma^d minus facets; both lists sorted */
    ivec freev = {0};
    int64_t fi = 0;
    for (int64_t t = 0; t < sigma->n; t++) {
        const int32_t *v = sigma->v + (d + 1) * t;
        while (fi < F->n && cmp_tuple(F->v + (d + 1) * fi, v, d + 1) < 0) fi++;
        if (fi < F->n && cmp_tuple(F->v + (d + 1) * fi, v, d + 1) == 0) continue;
        for (int k = 0; k <= d; k++) iv_push(&freev, v[k]);
    }
    slist free_s = take(&freev, d + 1);
    ivec flags = {0};
    int rc = ac2_flags(pr, &free_s, d, &flags);
    if (rc) return rc;
    ivec out = {0};
    for (int64_t t = 0; t < F->n; t++)
        for (int k = 0; k <= d; k++) iv_push(&out, F->v[(d + 1) * t + k]);
    for (int64_t t = 0; t < free_s.n; t++)
        if (flags.v[t])
            for (int k = 0; k <= d; k++) iv_push(&out, free_s.v[(d + 1) * t + k]);
    iv_free(&flags);
    free(free_s.v);
    K->v = out.v;
    K->n = sort_unique(out.v, out.n / (d + 1), d + 1);
    return OR_OK;
}

static long double to_ld(i128 x) {
    /* exact split into two 64-bit halves, then one rounding in long double */
    int neg = x < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    long double r = (long double)hi * 18446744073709551616.0L + (long double)lo;
    return neg ? -r : r;
}

static double orthosize_A2(const geom *s) {
    long double v = to_ld(s->os_num) / to_ld(s->os_den);
    return (double)(v / 1048576.0L);
}

/* ------------------------------------------------------------------ */
/* public entry points                                                  */

static void free_problem(problem *pr) {
    if (!pr) return;
    free(pr->P);
    free(pr->W);
    free(pr->nb_off);
    free(pr->nb);
    free(pr);
}

void oracle_free(oracle_result *r) {
    if (!r) return;
    for (int d = 0; d < 4; d++) {
        free(r->sigma[d].v);
        free(r->K[d].v);
        free(r->attached[d]);
        free(r->f[d]);
        free(r->orthosize[d]);
        free(r->src_dim[d]);
        free(r->src_idx[d]);
    }
    free_problem(r->prob);
    free(r);
}

int oracle_run(const double *centres, const double *radii, int64_t n, double alpha, int alpha_inf, int nthreads,
               oracle_result **out) {
    if (!out || n < 0 || (n > 0 && (!centres || !radii)) || n > 2000000000LL) return OR_ERR_ARG;
    *out = NULL;
    oracle_result *r = (oracle_result *)calloc(1, sizeof(oracle_result));
    problem *pr = (problem *)calloc(1, sizeof(problem));
    if (!r || !pr) {
        free(r);
        free(pr);
        return OR_ERR_OOM;
    }
    r->prob = pr;
    r->n_atoms = n;
    pr->n = n;
    pr->nthreads = nthreads;
    pr->inf = alpha_inf ? 1 : 0;
    pr->P = (int64_t *)malloc((size_t)(3 * n + 1) * sizeof(int64_t));
    pr->W = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!pr->P || !pr->W) {
        oracle_free(r);
        return OR_ERR_OOM;
    }
    /* quantise */
    int64_t wmax = 0;
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < 3; c++) {
            double x = centres[3 * i + c];
            if (!isfinite(x) || fabs(x) > 1048576.0) {
                oracle_free(r);
                return isfinite(x) ? OR_ERR_RANGE : OR_ERR_ARG;
            }
            pr->P[3 * i + c] = (int64_t)nearbyint(x * 1024.0);
        }
        double rr = radii[i];
        if (!isfinite(rr) || !(rr > 0)) {
            oracle_free(r);
            return OR_ERR_ARG;
        }
        int64_t R = (int64_t)nearbyint(rr * 1024.0);
        if (R < 1 || R * R > WEIGHT_LIMIT) {
            oracle_free(r);
            return OR_ERR_RANGE;
        }
        pr->W[i] = R * R;
        if (pr->W[i] > wmax) wmax = pr->W[i];
    }
    if (!pr->inf) {
        if (!isfinite(alpha) || fabs(alpha) * 1048576.0 > (double)WEIGHT_LIMIT) {
            oracle_free(r);
            return isfinite(alpha) ? OR_ERR_RANGE : OR_ERR_ARG;
        }
        pr->A = (int64_t)nearbyint(alpha * 1048576.0);
        pr->H2 = wmax + pr->A;
    }
    int rc = OR_OK;
    if (!pr->inf && pr->H2 <= 0 && n > 0) {
        /* no grown ball has positive radius: every list is empty */
        *out = r;
        for (int d = 0; d < 4; d++) {
            r->attached[d] = (uint8_t *)malloc(1);
            r->f[d] = (double *)malloc(sizeof(double));
            r->orthosize[d] = (double *)malloc(sizeof(double));
            r->src_dim[d] = (int32_t *)malloc(sizeof(int32_t));
            r->src_idx[d] = (int64_t *)malloc(sizeof(int64_t));
        }
        return OR_OK;
    }
    if (!pr->inf && 4 * pr->H2 > 4 * WEIGHT_LIMIT) {
        oracle_free(r);
        return OR_ERR_RANGE;
    }
    rc = build_neighbours(pr);
    if (rc) {
        oracle_free(r);
        return rc;
    }

    /* Step 1 */
    {
        ivec s0 = {0};
        for (int64_t i = 0; i < n; i++)
            if (pr->inf || -pr->W[i] <= pr->A) iv_push(&s0, (int32_t)i);
        r->sigma[0] = take(&s0, 1);
    }
    ivec tmp = {0};
    rc = parallel_collect(pr, n, NULL, body_sigma1, &tmp);
    if (rc) goto fail;
    r->sigma[1] = take(&tmp, 2);
    int64_t *up_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!up_off) {
        rc = OR_ERR_OOM;
        goto fail;
    }
    for (int64_t t = 0; t < r->sigma[1].n; t++) up_off[r->sigma[1].v[2 * t] + 1]++;
    for (int64_t i = 0; i < n; i++) up_off[i + 1] += up_off[i];
    int32_t *up = (int32_t *)malloc((size_t)(r->sigma[1].n + 1) * sizeof(int32_t));
    if (!up) {
        free(up_off);
        rc = OR_ERR_OOM;
        goto fail;
    }
    for (int64_t t = 0; t < r->sigma[1].n; t++) up[t] = r->sigma[1].v[2 * t + 1]; /* sorted by (i, j) */
    s1ctx c1 = {up_off, up, NULL};
    rc = parallel_collect(pr, n, &c1, body_sigma2, &tmp);
    if (rc) {
        free(up_off);
        free(up);
        goto fail;
    }
    r->sigma[2] = take(&tmp, 3);
    c1.s2 = &r->sigma[2];
    rc = parallel_collect(pr, r->sigma[2].n, &c1, body_sigma3, &tmp);
    free(up_off);
    free(up);
    if (rc) goto fail;
    r->sigma[3] = take(&tmp, 4);
    if (pr->range_error) {
        rc = OR_ERR_RANGE;
        goto fail;
    }

    /* Step 2 */
    {
        ivec flags = {0};
        rc = ac2_flags(pr, &r->sigma[3], 3, &flags);
        if (rc) goto fail;
        ivec k3 = {0};
        for (int64_t t = 0; t < r->sigma[3].n; t++)
            if (flags.v[t])
                for (int k = 0; k < 4; k++) iv_push(&k3, r->sigma[3].v[4 * t + k]);
        iv_free(&flags);
        r->K[3] = take(&k3, 4);
    }
    /* Steps 3, 4, 5 */
    for (int d = 2; d >= 0; d--) {
        slist F;
        if (d >= 1) {
            F = facets_of(&r->K[d + 1], d + 1);
        } else {
            ivec ends = {0};
            for (int64_t t = 0; t < 2 * r->K[1].n; t++) iv_push(&ends, r->K[1].v[t]);
            F.v = ends.v;
            F.n = sort_unique(ends.v, ends.n, 1);
        }
        rc = step_lower(pr, &r->sigma[d], &F, d, &r->K[d]);
        free(F.v);
        if (rc) goto fail;
    }
    if (pr->range_error) {
        rc = OR_ERR_RANGE;
        goto fail;
    }

    /* filtration: Size, top-down */
    for (int d = 3; d >= 0; d--) {
        int64_t m = r->K[d].n;
        r->attached[d] = (uint8_t *)malloc((size_t)(m ? m : 1));
        r->f[d] = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
        r->orthosize[d] = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
        r->src_dim[d] = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
        r->src_idx[d] = (int64_t *)malloc((size_t)(m ? m : 1) * sizeof(int64_t));
        if (!r->attached[d] || !r->f[d] || !r->orthosize[d] || !r->src_dim[d] || !r->src_idx[d]) {
            rc = OR_ERR_OOM;
            goto fail;
        }
        ivec flags = {0};
        if (d == 3) {
            for (int64_t t = 0; t < m; t++) iv_push(&flags, 1);
        } else {
            rc = ac2_flags(pr, &r->K[d], d, &flags);
            if (rc) goto fail;
        }
        for (int64_t t = 0; t < m; t++) {
            geom s;
            simplex_geom(pr, r->K[d].v + (d + 1) * t, d, &s);
            r->orthosize[d][t] = orthosize_A2(&s);
            r->attached[d][t] = flags.v[t] ? 0 : 1;
            r->f[d][t] = INFINITY;
            r->src_dim[d][t] = d;
            r->src_idx[d][t] = t;
            if (!r->attached[d][t]) r->f[d][t] = r->orthosize[d][t];
        }
        iv_free(&flags);
        if (d < 3) {
            /* attached: min over cofaces in K^{d+1}; lexicographically first coface wins ties */
            const slist *C = &r->K[d + 1];
            for (int64_t t = 0; t < C->n; t++) {
                const int32_t *v = C->v + (d + 2) * t;
                for (int drop = 0; drop <= d + 1; drop++) {
                    int32_t face[4];
                    int w = 0;
                    for (int k = 0; k <= d + 1; k++)
                        if (k != drop) face[w++] = v[k];
                    int64_t idx = find_tuple(&r->K[d], d, face);
                    if (idx < 0 || !r->attached[d][idx]) continue;
                    double fc = r->f[d + 1][t];
                    if (fc < r->f[d][idx]) {
                        r->f[d][idx] = fc;
                        r->src_dim[d][idx] = r->src_dim[d + 1][t];
                        r->src_idx[d][idx] = r->src_idx[d + 1][t];
                    }
                }
            }
        }
    }
    *out = r;
    return OR_OK;
fail:
    iv_free(&tmp);
    oracle_free(r);
    return rc;
}

int64_t oracle_count(const oracle_result *r, int what, int d) {
    if (!r || d < 0 || d > 3) return -1;
    return what == 0 ? r->K[d].n : r->sigma[d].n;
}

void oracle_copy_simplices(const oracle_result *r, int what, int d, int32_t *out) {
    const slist *L = what == 0 ? &r->K[d] : &r->sigma[d];
    if (L->n) memcpy(out, L->v, (size_t)L->n * (d + 1) * sizeof(int32_t));
}

void oracle_copy_values(const oracle_result *r, int d, double *f, double *orthosize, uint8_t *attached,
                        int32_t *src_dim, int64_t *src_idx) {
    int64_t m = r->K[d].n;
    if (!m) return;
    if (f) memcpy(f, r->f[d], (size_t)m * sizeof(double));
    if (orthosize) memcpy(orthosize, r->orthosize[d], (size_t)m * sizeof(double));
    if (attached) memcpy(attached, r->attached[d], (size_t)m);
    if (src_dim) memcpy(src_dim, r->src_dim[d], (size_t)m * sizeof(int32_t));
    if (src_idx) memcpy(src_idx, r->src_idx[d], (size_t)m * sizeof(int64_t));
}

/*
 * Closed-form gradient of L = sum_sigma w_sigma f_sigma with the combinatorics
 * fixed. f_sigma is the OrthoSize of its source simplex s. The orthocentre c
 * of s minimises pi(., b_v0) on the equal-power affine set; by the envelope
 * theorem with multipliers equal to the barycentric coordinates lambda_k of c
 * in aff(s): dOrthoSize/dp_k = 2 lambda_k (p_k - c), dOrthoSize/dr_k =
 * -2 r_k lambda_k. Evaluated from exact rationals, accumulated in double.
 * dldf[d] holds one weight per simplex of K^d (NULL = zero weights).
 */
int oracle_gradient(const oracle_result *r, const double *const *dldf, double *dldc, double *dldr) {
    problem *pr = r->prob;
    int64_t n = r->n_atoms;
    memset(dldc, 0, (size_t)(3 * n) * sizeof(double));
    memset(dldr, 0, (size_t)n * sizeof(double));
    for (int d = 0; d < 4; d++) {
        if (!dldf[d]) continue;
        for (int64_t t = 0; t < r->K[d].n; t++) {
            double w = dldf[d][t];
            if (w == 0.0) continue;
            int sd = r->src_dim[d][t];
            const int32_t *v = r->K[sd].v + (sd + 1) * r->src_idx[d][t];
            geom s;
            if (!simplex_geom(pr, v, sd, &s)) return OR_ERR_DEGENERATE;
            /* lambda_k = mu_k = nv_k / (2g) for k >= 1, lambda_0 = 1 - sum; y = ynum / (2g) */
            long double two_g = 2.0L * to_ld(s.g);
            long double lam[4], y[3];
            lam[0] = 1.0L;
            for (int k = 0; k < sd; k++) lam[k + 1] = to_ld(s.nv[k]) / two_g;
            if (sd > 0) {
                /* 1 - sum nv / 2g, formed exactly */
                i128 tot = 0;
                for (int k = 0; k < sd; k++) tot += s.nv[k];
                lam[0] = to_ld(2 * s.g - tot) / two_g;
            }
            for (int c = 0; c < 3; c++) y[c] = sd > 0 ? to_ld(s.ynum[c]) / two_g : 0.0L;
            for (int k = 0; k <= sd; k++) {
                int32_t a = v[k];
                for (int c = 0; c < 3; c++) {
                    long double qk = k == 0 ? 0.0L : (long double)s.q[k - 1][c];
                    /* p_k - c = q_k - y, in A */
                    dldc[3 * a + c] += (double)((long double)w * 2.0L * lam[k] * (qk - y[c]) / 1024.0L);
                }
                long double rk = sqrtl((long double)pr->W[a]) / 1024.0L;
                dldr[a] += (double)((long double)w * -2.0L * rk * lam[k]);
            }
        }
    }
    return OR_OK;
}
