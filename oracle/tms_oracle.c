/*
 * CPU oracle for the mesh-vs-mesh intersection search -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct FP64 reference of what the search computes.
 * It is linked only by tests, by the package's smoke check and by the benchmark's
 * CPU-baseline leg; the product search path never calls it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off: no fused multiply-add, so every product and sum is rounded
 * separately, as written).
 *
 * What it follows (arXiv 2109.14814):
 *   - mesh and triangle definitions: Sec. 6.1 (vertex grid, quads Q_ik with the
 *     theta index taken modulo N) and Sec. 6.2 (triangles T1, T2 of each quad);
 *   - the narrow-phase test: Sec. 6.2.4, Eq. (precise): solve
 *       x2 + (x1 - x2) a + (x3 - x2) b = y2 + (y1 - y2) c + (y3 - y2) d
 *     for (a, b, c, d); the triangles meet iff a, b, c, d >= 0, a + b <= 1 and
 *     c + d <= 1, and the common point is either side of the equation;
 *   - the (theta, s) estimates from (a, b) and (c, d): Sec. 6.2.4, the four
 *     interpolation formulas that follow Eq. (precise), with the vertex orderings
 *     x1, x2, x3 (and y1, y2, y3) given there;
 *   - the bounding-box test used for exact pruning: Sec. 6.2.2
 *     (two boxes are disjoint iff some coordinate's max of one is below the
 *     other's min); a triangle lies inside its box, so pruning by closed box
 *     overlap never removes an intersecting pair.
 * Readings where the paper is silent (tolerance tau, singular systems, the
 * normalised-column determinant rho as the degeneracy measure, the periodic
 * neighbour i+1 mod N) are listed in the repository's design notes.
 *
 * The 4x4 system is solved by textbook Gaussian elimination with partial
 * pivoting (pivot = largest |entry| in the column, ties to the lowest row),
 * followed by back substitution.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559

typedef struct {
    const double *X;   /* 4*M*N: coordinate c of vertex (i, k) at X[c*M*N + k*N + i] */
    const double *s;   /* M values s_k, increasing */
    int N, M;
    int periodic;      /* 1: quads i = 0..N-1 (i+1 taken mod N); 0: i = 0..N-2 */
} omesh;

typedef struct {
    long long triA, triB;
    double z[4];        /* a, b, c, d */
    double P[4];        /* x-side point x2 + a(x1-x2) + b(x3-x2) */
    double params[4];   /* theta_u, s_u, theta_s, s_s */
    double rho;         /* |det| / prod of column norms */
    double margin;      /* min(a, b, c, d, 1-a-b, 1-c-d) */
    double det;
    double gap;         /* |x-side point - y-side point|_inf (diagnostic) */
    int hit;
    int singular;
} oracle_rec;

/* ---------------------------------------------------------------------- */
/* mesh enumeration (Sec. 6.1, Sec. 6.2)                                   */
/* ---------------------------------------------------------------------- */

static long long n_tri_ids(const omesh *m) { return 2LL * m->N * (m->M - 1); }

static int tri_valid(const omesh *m, long long t) {
    if (t < 0 || t >= n_tri_ids(m)) return 0;
    long long q = t / 2;
    int i = (int)(q % m->N);
    return m->periodic || i < m->N - 1;
}

static void vertex(const omesh *m, int i, int k, double v[4]) {
    long long MN = (long long)m->M * m->N;
    for (int c = 0; c < 4; c++) v[c] = m->X[c * MN + (long long)k * m->N + i];
}

/* grid indices of (x1, x2, x3) of triangle t:
 *   T1 (tau 0): x1 = W(i+1, k), x2 = W(i, k),     x3 = W(i, k+1)
 *   T2 (tau 1): x1 = W(i, k+1), x2 = W(i+1, k+1), x3 = W(i+1, k)   */
static void tri_ij(const omesh *m, long long t, int ii[3], int kk[3]) {
    long long q = t / 2;
    int tau = (int)(t % 2);
    int i = (int)(q % m->N), k = (int)(q / m->N);
    int ip = (i + 1) % m->N;
    if (tau == 0) {
        ii[0] = ip; kk[0] = k;
        ii[1] = i;  kk[1] = k;
        ii[2] = i;  kk[2] = k + 1;
    } else {
        ii[0] = i;  kk[0] = k + 1;
        ii[1] = ip; kk[1] = k + 1;
        ii[2] = ip; kk[2] = k;
    }
}

static void tri_vertices(const omesh *m, long long t, double v[3][4]) {
    int ii[3], kk[3];
    tri_ij(m, t, ii, kk);
    for (int j = 0; j < 3; j++) vertex(m, ii[j], kk[j], v[j]);
}

/* (theta, s) estimate for weights (a, b) in triangle t (the formulas that follow
 * Eq. (precise)); theta_{i+1} is theta_i + dtheta (not wrapped), then the result
 * is wrapped into [0, 2 pi). */
static void tri_params(const omesh *m, long long t, double a, double b, double out[2]) {
    long long q = t / 2;
    int tau = (int)(t % 2);
    int i = (int)(q % m->N), k = (int)(q / m->N);
    double dth = TWO_PI / m->N;
    double th_i = i * dth, th_ip = th_i + dth;
    double s_k = m->s[k], s_kp = m->s[k + 1];
    double th, sv;
    if (tau == 0) {
        th = (1.0 - a) * th_i + a * th_ip;
        sv = (1.0 - b) * s_k + b * s_kp;
    } else {
        th = a * th_i + (1.0 - a) * th_ip;
        sv = b * s_k + (1.0 - b) * s_kp;
    }
    th = fmod(th, TWO_PI);
    if (th < 0) th += TWO_PI;
    out[0] = th;
    out[1] = sv;
}

/* ---------------------------------------------------------------------- */
/* Gaussian elimination with partial pivoting on a 4x4 system               */
/* ---------------------------------------------------------------------- */

/* Solves A z = r.  A is row-major A[row][col] and is overwritten.  Returns 1 on
 * success, 0 when a pivot is exactly zero (singular).  *det receives the
 * determinant (sign of the row swaps times the product of the pivots). */
int oracle_solve4(double A[4][4], double r[4], double z[4], double *det) {
    double sign = 1.0;
    for (int col = 0; col < 4; col++) {
        int p = col;
        double best = fabs(A[col][col]);
        for (int row = col + 1; row < 4; row++) {
            if (fabs(A[row][col]) > best) { best = fabs(A[row][col]); p = row; }
        }
        if (best == 0.0) { *det = 0.0; return 0; }
        if (p != col) {
            for (int j = 0; j < 4; j++) { double t = A[p][j]; A[p][j] = A[col][j]; A[col][j] = t; }
            double t = r[p]; r[p] = r[col]; r[col] = t;
            sign = -sign;
        }
        for (int row = col + 1; row < 4; row++) {
            double f = A[row][col] / A[col][col];
            A[row][col] = 0.0;
            for (int j = col + 1; j < 4; j++) A[row][j] = A[row][j] - f * A[col][j];
            r[row] = r[row] - f * r[col];
        }
    }
    for (int row = 3; row >= 0; row--) {
        double acc = r[row];
        for (int j = row + 1; j < 4; j++) acc = acc - A[row][j] * z[j];
        z[row] = acc / A[row][row];
    }
    double d = sign;
    for (int j = 0; j < 4; j++) d = d * A[j][j];
    *det = d;
    return 1;
}

/* flat wrapper for testing the solver on its own: A row-major 16 values */
int oracle_solve4_flat(const double *A16, const double *r4, double *z4, double *det) {
    double A[4][4], r[4];
    for (int i = 0; i < 4; i++) { r[i] = r4[i]; for (int j = 0; j < 4; j++) A[i][j] = A16[4 * i + j]; }
    return oracle_solve4(A, r, z4, det);
}

/* ---------------------------------------------------------------------- */
/* narrow phase for one triangle pair (Sec. 6.2.4, Eq. (precise))           */
/* ---------------------------------------------------------------------- */

static double min6(double a, double b, double c, double d, double e, double f) {
    double m = a;
    if (b < m) m = b;
    if (c < m) m = c;
    if (d < m) m = d;
    if (e < m) m = e;
    if (f < m) m = f;
    return m;
}

/* Columns of the system matrix: x1-x2, x3-x2, y2-y1, y2-y3; right side y2-x2.
 * (Moving the unknown terms of Eq. (precise) to the left gives exactly this.) */
static void build_system(const double x[3][4], const double y[3][4], double A[4][4], double r[4]) {
    for (int c = 0; c < 4; c++) {
        A[c][0] = x[0][c] - x[1][c];
        A[c][1] = x[2][c] - x[1][c];
        A[c][2] = y[1][c] - y[0][c];
        A[c][3] = y[1][c] - y[2][c];
        r[c] = y[1][c] - x[1][c];
    }
}

static void eval_pair(const double x[3][4], const double y[3][4], double tau, oracle_rec *o) {
    double A[4][4], r[4], z[4] = {0, 0, 0, 0}, det = 0.0;
    build_system(x, y, A, r);
    double norm_prod = 1.0;
    for (int j = 0; j < 4; j++) {
        double ss = 0.0;
        for (int c = 0; c < 4; c++) ss = ss + A[c][j] * A[c][j];
        norm_prod = norm_prod * sqrt(ss);
    }
    int ok = oracle_solve4(A, r, z, &det);
    o->det = det;
    o->singular = !ok;
    o->rho = (norm_prod > 0.0) ? fabs(det) / norm_prod : 0.0;
    for (int j = 0; j < 4; j++) o->z[j] = ok ? z[j] : NAN;
    if (!ok) {
        o->margin = -INFINITY;
        o->hit = 0;
        for (int c = 0; c < 4; c++) o->P[c] = NAN;
        o->gap = NAN;
        return;
    }
    double a = z[0], b = z[1], c = z[2], d = z[3];
    o->margin = min6(a, b, c, d, 1.0 - a - b, 1.0 - c - d);
    int finite = isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
    o->hit = finite && (o->rho > 0.0) && (o->margin >= -tau);
    double gap = 0.0;
    for (int k = 0; k < 4; k++) {
        double px = x[1][k] + a * (x[0][k] - x[1][k]) + b * (x[2][k] - x[1][k]);
        double py = y[1][k] + c * (y[0][k] - y[1][k]) + d * (y[2][k] - y[1][k]);
        o->P[k] = px;
        double g = fabs(px - py);
        if (g > gap) gap = g;
    }
    o->gap = gap;
}

static void eval_mesh_pair(const omesh *ma, const omesh *mb, long long ta, long long tb,
                           double tau, oracle_rec *o) {
    double x[3][4], y[3][4];
    tri_vertices(ma, ta, x);
    tri_vertices(mb, tb, y);
    eval_pair(x, y, tau, o);
    o->triA = ta;
    o->triB = tb;
    if (o->hit || !o->singular) {
        double pu[2], ps[2];
        tri_params(ma, ta, o->z[0], o->z[1], pu);
        tri_params(mb, tb, o->z[2], o->z[3], ps);
        o->params[0] = pu[0]; o->params[1] = pu[1];
        o->params[2] = ps[0]; o->params[3] = ps[1];
    } else {
        for (int j = 0; j < 4; j++) o->params[j] = NAN;
    }
}

/* ---------------------------------------------------------------------- */
/* exported: single pair / raw triangles                                    */
/* ---------------------------------------------------------------------- */

static omesh mk(const double *X, const double *s, int N, int M, int periodic) {
    omesh m;
    m.X = X; m.s = s; m.N = N; m.M = M; m.periodic = periodic;
    return m;
}

/* Evaluate the narrow-phase test for explicit vertices x[3][4], y[3][4]. */
void oracle_tri_pair(const double *x12, const double *y12, double tau, oracle_rec *out) {
    double x[3][4], y[3][4];
    for (int j = 0; j < 3; j++)
        for (int c = 0; c < 4; c++) { x[j][c] = x12[4 * j + c]; y[j][c] = y12[4 * j + c]; }
    memset(out, 0, sizeof(*out));
    eval_pair(x, y, tau, out);
    out->triA = -1; out->triB = -1;
    for (int j = 0; j < 4; j++) out->params[j] = NAN;
}

/* Evaluate a list of (triA, triB) pairs of two meshes. */
void oracle_eval_pairs(const double *XA, const double *sA, int NA, int MA, int perA,
                       const double *XB, const double *sB, int NB, int MB, int perB,
                       const long long *triA, const long long *triB, long long n,
                       double tau, oracle_rec *out) {
    omesh ma = mk(XA, sA, NA, MA, perA), mb = mk(XB, sB, NB, MB, perB);
    #pragma omp parallel for schedule(static)
    for (long long h = 0; h < n; h++) {
        memset(&out[h], 0, sizeof(oracle_rec));
        if (!tri_valid(&ma, triA[h]) || !tri_valid(&mb, triB[h])) {
            out[h].triA = triA[h]; out[h].triB = triB[h]; out[h].singular = 1;
            out[h].margin = -INFINITY;
            continue;
        }
        eval_mesh_pair(&ma, &mb, triA[h], triB[h], tau, &out[h]);
    }
}

/* Vertex coordinates of triangles (x1, x2, x3), 12 doubles per triangle. */
void oracle_tri_coords(const double *X, const double *s, int N, int M, int periodic,
                       const long long *tri, long long n, double *out12) {
    omesh m = mk(X, s, N, M, periodic);
    for (long long h = 0; h < n; h++) {
        double v[3][4];
        tri_vertices(&m, tri[h], v);
        for (int j = 0; j < 3; j++)
            for (int c = 0; c < 4; c++) out12[12 * h + 4 * j + c] = v[j][c];
    }
}

/* ---------------------------------------------------------------------- */
/* all-pairs brute force                                                    */
/* ---------------------------------------------------------------------- */

static void push_hit(oracle_rec *out, long long cap, long long *count, const oracle_rec *o) {
    long long idx;
    #pragma omp atomic capture
    idx = (*count)++;
    if (idx < cap) out[idx] = *o;
}

/* Every pair (tA, tB) of valid triangles is tested.  Returns the number of hits
 * (raw, before any merging); at most cap records are written, in no order. */
long long oracle_bruteforce(const double *XA, const double *sA, int NA, int MA, int perA,
                            const double *XB, const double *sB, int NB, int MB, int perB,
                            double tau, oracle_rec *out, long long cap) {
    omesh ma = mk(XA, sA, NA, MA, perA), mb = mk(XB, sB, NB, MB, perB);
    long long TA = n_tri_ids(&ma), TB = n_tri_ids(&mb);
    long long count = 0;
    #pragma omp parallel for schedule(dynamic, 16)
    for (long long ta = 0; ta < TA; ta++) {
        if (!tri_valid(&ma, ta)) continue;
        double x[3][4];
        tri_vertices(&ma, ta, x);
        for (long long tb = 0; tb < TB; tb++) {
            if (!tri_valid(&mb, tb)) continue;
            double y[3][4];
            tri_vertices(&mb, tb, y);
            oracle_rec o;
            eval_pair(x, y, tau, &o);
            if (o.hit) {
                o.triA = ta; o.triB = tb;
                double pu[2], ps[2];
                tri_params(&ma, ta, o.z[0], o.z[1], pu);
                tri_params(&mb, tb, o.z[2], o.z[3], ps);
                o.params[0] = pu[0]; o.params[1] = pu[1];
                o.params[2] = ps[0]; o.params[3] = ps[1];
                push_hit(out, cap, &count, &o);
            }
        }
    }
    return count;
}

/* ---------------------------------------------------------------------- */
/* exact pruning by closed bounding-box overlap                             */
/* ---------------------------------------------------------------------- */

typedef struct { double lo[4], hi[4]; } box4;

static void tri_box(const omesh *m, long long t, box4 *b) {
    double v[3][4];
    tri_vertices(m, t, v);
    for (int c = 0; c < 4; c++) {
        double lo = v[0][c], hi = v[0][c];
        for (int j = 1; j < 3; j++) {
            if (v[j][c] < lo) lo = v[j][c];
            if (v[j][c] > hi) hi = v[j][c];
        }
        b->lo[c] = lo; b->hi[c] = hi;
    }
}

/* closed overlap: disjoint iff some max of one box is below the other's min */
static int boxes_overlap(const box4 *a, const box4 *b) {
    for (int c = 0; c < 4; c++) {
        if (a->hi[c] < b->lo[c] || b->hi[c] < a->lo[c]) return 0;
    }
    return 1;
}

/* A bounding-volume hierarchy over the B triangles: each node's box contains
 * the boxes of all triangles below it, so a query box that misses a node's box
 * misses every triangle below it.  Built by recursive median split of the
 * triangle centroids along the widest axis; leaves hold at most 8 triangles. */
typedef struct {
    box4 box;
    long long start, count;    /* leaf range in ids[] */
    int left, right;           /* children (-1 for a leaf) */
} bnode;

typedef struct {
    box4 *boxB;                /* indexed by triangle id */
    long long *ids;            /* valid B triangle ids, permuted by the build */
    long long nB;
    bnode *nodes;
    int n_nodes, cap_nodes;
} bvh;

static double centroid(const box4 *b, int axis) { return 0.5 * (b->lo[axis] + b->hi[axis]); }

/* partial sort: ids[lo..hi) rearranged so that position kth holds the element of
 * rank kth by centroid along axis (quickselect, Hoare partition) */
static void select_kth(const box4 *boxes, long long *ids, long long lo, long long hi,
                       long long kth, int axis) {
    while (hi - lo > 1) {
        double pivot = centroid(&boxes[ids[lo + (hi - lo) / 2]], axis);
        long long i = lo, j = hi - 1;
        while (i <= j) {
            while (centroid(&boxes[ids[i]], axis) < pivot) i++;
            while (centroid(&boxes[ids[j]], axis) > pivot) j--;
            if (i <= j) { long long t = ids[i]; ids[i] = ids[j]; ids[j] = t; i++; j--; }
        }
        if (kth <= j) hi = j + 1;
        else if (kth >= i) lo = i;
        else return;
    }
}

static int bvh_build(bvh *h, long long start, long long count) {
    if (h->n_nodes == h->cap_nodes) {
        h->cap_nodes *= 2;
        h->nodes = (bnode *)realloc(h->nodes, sizeof(bnode) * (size_t)h->cap_nodes);
    }
    int me = h->n_nodes++;
    box4 b = h->boxB[h->ids[start]];
    double clo[4], chi[4];
    for (int c = 0; c < 4; c++) clo[c] = chi[c] = centroid(&b, c);
    for (long long j = start; j < start + count; j++) {
        const box4 *t = &h->boxB[h->ids[j]];
        for (int c = 0; c < 4; c++) {
            if (t->lo[c] < b.lo[c]) b.lo[c] = t->lo[c];
            if (t->hi[c] > b.hi[c]) b.hi[c] = t->hi[c];
            double m = centroid(t, c);
            if (m < clo[c]) clo[c] = m;
            if (m > chi[c]) chi[c] = m;
        }
    }
    h->nodes[me].box = b;
    h->nodes[me].start = start;
    h->nodes[me].count = count;
    h->nodes[me].left = h->nodes[me].right = -1;
    if (count <= 8) return me;
    int axis = 0;
    for (int c = 1; c < 4; c++) if (chi[c] - clo[c] > chi[axis] - clo[axis]) axis = c;
    long long half = count / 2;
    select_kth(h->boxB, h->ids, start, start + count, start + half, axis);
    int l = bvh_build(h, start, half);
    int r = bvh_build(h, start + half, count - half);
    h->nodes[me].left = l;
    h->nodes[me].right = r;
    return me;
}

static void bvh_prepare(const omesh *mb, bvh *h) {
    long long TB = n_tri_ids(mb);
    h->boxB = (box4 *)malloc(sizeof(box4) * (size_t)(TB > 0 ? TB : 1));
    h->ids = (long long *)malloc(sizeof(long long) * (size_t)(TB > 0 ? TB : 1));
    long long n = 0;
    for (long long t = 0; t < TB; t++) {
        if (!tri_valid(mb, t)) continue;
        tri_box(mb, t, &h->boxB[t]);
        h->ids[n++] = t;
    }
    h->nB = n;
    h->cap_nodes = 1024;
    h->n_nodes = 0;
    h->nodes = (bnode *)malloc(sizeof(bnode) * (size_t)h->cap_nodes);
    if (n > 0) bvh_build(h, 0, n);
}

static void bvh_free(bvh *h) { free(h->boxB); free(h->ids); free(h->nodes); }

/* Visit every B triangle whose closed box overlaps box qa; calls back per pair. */
typedef void (*pair_fn)(long long tb, void *ctx);

static void bvh_query(const bvh *h, const box4 *qa, pair_fn fn, void *ctx) {
    if (h->n_nodes == 0) return;
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const bnode *nd = &h->nodes[stack[--sp]];
        if (!boxes_overlap(qa, &nd->box)) continue;
        if (nd->left < 0) {
            for (long long j = nd->start; j < nd->start + nd->count; j++) {
                long long tb = h->ids[j];
                if (boxes_overlap(qa, &h->boxB[tb])) fn(tb, ctx);
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
}

typedef struct {
    const omesh *ma, *mb;
    long long ta;
    double x[3][4];
    double tau;
    oracle_rec *out;
    long long cap;
    long long *count;
    long long n_overlap;
    int want_hits;
    long long *pairs;
} qctx;

static void on_pair(long long tb, void *p) {
    qctx *q = (qctx *)p;
    q->n_overlap++;
    if (q->pairs) {
        long long idx;
        #pragma omp atomic capture
        idx = (*q->count)++;
        if (idx < q->cap) { q->pairs[2 * idx] = q->ta; q->pairs[2 * idx + 1] = tb; }
        return;
    }
    if (!q->want_hits) return;
    double y[3][4];
    tri_vertices(q->mb, tb, y);
    oracle_rec o;
    eval_pair(q->x, y, q->tau, &o);
    if (o.hit) {
        o.triA = q->ta; o.triB = tb;
        double pu[2], ps[2];
        tri_params(q->ma, q->ta, o.z[0], o.z[1], pu);
        tri_params(q->mb, tb, o.z[2], o.z[3], ps);
        o.params[0] = pu[0]; o.params[1] = pu[1];
        o.params[2] = ps[0]; o.params[3] = ps[1];
        push_hit(q->out, q->cap, q->count, &o);
    }
}

static long long query_one(const omesh *ma, const omesh *mb, const bvh *h, long long ta,
                           double tau, oracle_rec *out, long long cap, long long *count,
                           long long *pairs) {
    qctx q;
    q.ma = ma; q.mb = mb; q.ta = ta; q.tau = tau; q.out = out; q.cap = cap;
    q.count = count; q.n_overlap = 0; q.want_hits = 1; q.pairs = pairs;
    tri_vertices(ma, ta, q.x);
    box4 ba;
    tri_box(ma, ta, &ba);
    bvh_query(h, &ba, on_pair, &q);
    return q.n_overlap;
}

/* All hits, visiting only pairs whose closed boxes overlap.  *n_overlap receives
 * the number of box-overlapping pairs.  Returns the raw hit count. */
long long oracle_pruned(const double *XA, const double *sA, int NA, int MA, int perA,
                        const double *XB, const double *sB, int NB, int MB, int perB,
                        double tau, oracle_rec *out, long long cap, long long *n_overlap) {
    omesh ma = mk(XA, sA, NA, MA, perA), mb = mk(XB, sB, NB, MB, perB);
    bvh h;
    bvh_prepare(&mb, &h);
    long long TA = n_tri_ids(&ma);
    long long count = 0, nov = 0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+:nov)
    for (long long ta = 0; ta < TA; ta++) {
        if (!tri_valid(&ma, ta)) continue;
        nov += query_one(&ma, &mb, &h, ta, tau, out, cap, &count, NULL);
    }
    bvh_free(&h);
    if (n_overlap) *n_overlap = nov;
    return count;
}

/* Hits of the listed A triangles against all of B (sampled parity at sizes
 * where the full oracle is too slow). */
long long oracle_hits_for_A(const double *XA, const double *sA, int NA, int MA, int perA,
                            const double *XB, const double *sB, int NB, int MB, int perB,
                            const long long *trisA, long long nA, double tau,
                            oracle_rec *out, long long cap) {
    omesh ma = mk(XA, sA, NA, MA, perA), mb = mk(XB, sB, NB, MB, perB);
    bvh h;
    bvh_prepare(&mb, &h);
    long long count = 0;
    #pragma omp parallel for schedule(dynamic, 4)
    for (long long j = 0; j < nA; j++) {
        if (!tri_valid(&ma, trisA[j])) continue;
        query_one(&ma, &mb, &h, trisA[j], tau, out, cap, &count, NULL);
    }
    bvh_free(&h);
    return count;
}

/* Closed box-overlap pairs (triA, triB), for checking that a broad phase keeps
 * all of them.  Returns the count; writes at most cap pairs. */
long long oracle_box_pairs(const double *XA, const double *sA, int NA, int MA, int perA,
                           const double *XB, const double *sB, int NB, int MB, int perB,
                           long long *pairs, long long cap) {
    omesh ma = mk(XA, sA, NA, MA, perA), mb = mk(XB, sB, NB, MB, perB);
    bvh h;
    bvh_prepare(&mb, &h);
    long long TA = n_tri_ids(&ma);
    long long count = 0;
    #pragma omp parallel for schedule(dynamic, 64)
    for (long long ta = 0; ta < TA; ta++) {
        if (!tri_valid(&ma, ta)) continue;
        query_one(&ma, &mb, &h, ta, 0.0, NULL, cap, &count, pairs);
    }
    bvh_free(&h);
    return count;
}

/* ---------------------------------------------------------------------- */
/* reverse-mode derivative of one hit                                       */
/* ---------------------------------------------------------------------- */

/* Given upstream gradients gP (on the x-side point P) and gz (on a, b, c, d),
 * returns the gradients on the six vertices x1, x2, x3, y1, y2, y3 (12 + 12).
 * Implicit differentiation of A z = r:  dz = A^{-1} (dr - dA z), so with
 * zbar = gz + (dP/dz)^T gP and w = A^{-T} zbar:  rbar = w,  Abar = -w z^T;
 * P = x2 + a(x1-x2) + b(x3-x2) also depends on x directly.
 * w is found with the same Gaussian elimination applied to A^T.
 * Returns 0 when the system is singular. */
int oracle_pair_grad(const double *x12, const double *y12, const double *gP, const double *gz,
                     double *gx12, double *gy12, double *z_out) {
    double x[3][4], y[3][4];
    for (int j = 0; j < 3; j++)
        for (int c = 0; c < 4; c++) { x[j][c] = x12[4 * j + c]; y[j][c] = y12[4 * j + c]; }
    double A[4][4], r[4], z[4], det;
    build_system(x, y, A, r);
    double At[4][4];
    for (int i = 0; i < 4; i++) for (int j = 0; j < 4; j++) At[i][j] = A[j][i];
    if (!oracle_solve4(A, r, z, &det)) return 0;
    double zbar[4];
    for (int j = 0; j < 4; j++) zbar[j] = gz[j];
    /* dP/da = x1 - x2, dP/db = x3 - x2 */
    for (int c = 0; c < 4; c++) {
        zbar[0] = zbar[0] + (x[0][c] - x[1][c]) * gP[c];
        zbar[1] = zbar[1] + (x[2][c] - x[1][c]) * gP[c];
    }
    double w[4];
    if (!oracle_solve4(At, zbar, w, &det)) return 0;
    /* Abar[:, j] = -z_j w; columns: x1-x2, x3-x2, y2-y1, y2-y3; rbar = w (r = y2 - x2) */
    double gx[3][4], gy[3][4];
    for (int c = 0; c < 4; c++) {
        double a = z[0], b = z[1], cc = z[2], d = z[3];
        gx[0][c] = -a * w[c];
        gx[1][c] = a * w[c] + b * w[c] - w[c];
        gx[2][c] = -b * w[c];
        gy[0][c] = cc * w[c];
        gy[1][c] = -cc * w[c] - d * w[c] + w[c];
        gy[2][c] = d * w[c];
        /* direct dependence of P on the vertices at fixed (a, b) */
        gx[0][c] = gx[0][c] + a * gP[c];
        gx[1][c] = gx[1][c] + (1.0 - a - b) * gP[c];
        gx[2][c] = gx[2][c] + b * gP[c];
    }
    for (int j = 0; j < 3; j++)
        for (int c = 0; c < 4; c++) { gx12[4 * j + c] = gx[j][c]; gy12[4 * j + c] = gy[j][c]; }
    for (int j = 0; j < 4; j++) z_out[j] = z[j];
    return 1;
}

int oracle_sizeof_rec(void) { return (int)sizeof(oracle_rec); }
