/*
 * vt_oracle.c -- plain, slow FP64 CPU Voronoi tessellator.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do. It shares no code, header, table or helper with the CUDA
 * path.
 *
 * What it computes (votess paper, Statement of need and Summary): the Voronoi
 * cell of generator p_i inside the domain box,
 *
 *     C_i = Box  intersect  { x : |x - p_i| <= |x - p_j|  for all j != i },
 *
 * obtained the way the Summary describes the cell-by-cell method: sort the
 * neighbours of p_i by distance (k nearest, here from a kd-tree), clip the
 * box by the perpendicular bisector plane of (p_i, p_j) for each neighbour
 * nearest first, and stop as soon as the "security radius" condition shows
 * that no farther generator can cut the cell. If the k listed neighbours do not
 * suffice, k is doubled and the cell is recomputed (the paper falls back to a
 * CPU path there; on the CPU the retry is the fallback).
 *
 * Representation: the polyhedron is a list of planar faces, each a vertex
 * loop (counter-clockwise seen from outside) tagged with the generator index
 * of its bisector (>= 0) or a wall id (-1..-6). A clip is Sutherland-Hodgman
 * on every face plus a new "cap" face made of the points on the cutting
 * plane, ordered by angle. All arithmetic is IEEE double with no contraction
 * (build with -ffp-contract=off) so results are identical on x86-64 and
 * aarch64 hosts.
 *
 * Readings where the paper is silent:
 *  - the bounding box is the non-periodic domain box (walls are clip planes);
 *  - the cell is computed in the local frame of p_i (coordinates p - p_i);
 *  - kNN order is (d2, index) with d2 = ((dx*dx + dy*dy) + dz*dz) in double
 *    from the float32 inputs, dx = (double)p_j.x - (double)p_i.x;
 *  - the security-radius test is non-strict: before clipping with neighbour
 *    m, the cell is final when 4 R^2 <= d2_m, R = max vertex distance from
 *    p_i; after all k neighbours, when 4 R^2 <= d2_{k-1}; when the list holds
 *    all n-1 other generators the cell is final by construction;
 *  - a vertex with s = n.v - b == 0 exactly lies on the plane and is kept;
 *  - j is reported as a neighbour when its face has area > 1e-12 V^(2/3).
 *
 * Periodic boxes (vto_tessellate_periodic, vto_knn_periodic): the same
 * definition with every generator repeated at all its images p_j + t L
 * (L = hi - lo, t integer); see the periodic section below.
 */
#include "vt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */

typedef struct { double x, y, z; } vec3;

static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vscale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(vec3 a, vec3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
static vec3 vcross(vec3 a, vec3 b)
{
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static int veq(vec3 a, vec3 b) { return a.x == b.x && a.y == b.y && a.z == b.z; }
/* det[a b c] = a . (b x c): six times the signed volume of tet (0, a, b, c) */
static double vdet(vec3 a, vec3 b, vec3 c) { return vdot(a, vcross(b, c)); }

/* squared distance, in the exact expression order the kNN key uses */
static double dist2_f32(const float* p, const float* q)
{
    double dx = (double)q[0] - (double)p[0];
    double dy = (double)q[1] - (double)p[1];
    double dz = (double)q[2] - (double)p[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* ------------------------------------------------------------------ */
/* kd-tree k-nearest-neighbour search (exact, ties by index)           */
/* ------------------------------------------------------------------ */

#define KD_LEAF 8

typedef struct {
    int64_t lo, hi;    /* range in the permutation */
    int axis;          /* -1 for a leaf */
    double split;      /* coordinate of the median point */
    int64_t left, right;
} kd_node;

struct vto_kdtree {
    const float* pts;
    int64_t n;
    int64_t* perm;
    kd_node* nodes;
    int64_t n_nodes, cap_nodes;
};

static double coord(const vto_kdtree* t, int64_t i, int axis) { return (double)t->pts[3 * i + axis]; }

/* order by (coordinate, index) so the median split is well defined */
static int kd_less(const vto_kdtree* t, int64_t a, int64_t b, int axis)
{
    double ca = coord(t, a, axis), cb = coord(t, b, axis);
    return ca < cb || (ca == cb && a < b);
}

/* quickselect: after the call perm[m] holds the element of rank m-lo in [lo, hi) */
static void kd_select(vto_kdtree* t, int64_t lo, int64_t hi, int64_t m, int axis)
{
    int64_t* p = t->perm;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t tmp = p[mid]; p[mid] = p[hi - 1]; p[hi - 1] = tmp; /* pivot to the end */
        int64_t pv = p[hi - 1], store = lo;
        for (int64_t i = lo; i < hi - 1; ++i)
            if (kd_less(t, p[i], pv, axis)) { tmp = p[i]; p[i] = p[store]; p[store] = tmp; ++store; }
        tmp = p[store]; p[store] = p[hi - 1]; p[hi - 1] = tmp;
        if (store == m) return;
        if (m < store) hi = store; else lo = store + 1;
    }
}

static int64_t kd_build_rec(vto_kdtree* t, int64_t lo, int64_t hi)
{
    if (t->n_nodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes * 2 + 16;
        t->nodes = (kd_node*)realloc(t->nodes, (size_t)t->cap_nodes * sizeof(kd_node));
    }
    int64_t id = t->n_nodes++;
    t->nodes[id].lo = lo; t->nodes[id].hi = hi;
    t->nodes[id].axis = -1; t->nodes[id].left = t->nodes[id].right = -1;
    if (hi - lo <= KD_LEAF) return id;
    /* split the widest extent at its median */
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = lo; i < hi; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = coord(t, t->perm[i], a);
            if (c < mn[a]) mn[a] = c;
            if (c > mx[a]) mx[a] = c;
        }
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (mx[a] - mn[a] > mx[axis] - mn[axis]) axis = a;
    int64_t m = lo + (hi - lo) / 2;
    kd_select(t, lo, hi, m, axis);
    t->nodes[id].axis = axis;
    t->nodes[id].split = coord(t, t->perm[m], axis);
    int64_t l = kd_build_rec(t, lo, m);
    int64_t r = kd_build_rec(t, m, hi);
    t->nodes[id].left = l; t->nodes[id].right = r;
    return id;
}

vto_kdtree* vto_kdtree_build(const float* pts, int64_t n)
{
    vto_kdtree* t = (vto_kdtree*)calloc(1, sizeof(vto_kdtree));
    t->pts = pts; t->n = n;
    t->perm = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    if (n > 0) kd_build_rec(t, 0, n);
    return t;
}

void vto_kdtree_free(vto_kdtree* t)
{
    if (!t) return;
    free(t->perm); free(t->nodes); free(t);
}

/* bounded max-heap of (d2, idx), ordered lexicographically */
typedef struct { double d2; int64_t idx; } kv;
static int kv_gt(kv a, kv b) { return a.d2 > b.d2 || (a.d2 == b.d2 && a.idx > b.idx); }

typedef struct { kv* h; int size, cap; } kheap;

static void kheap_push(kheap* H, kv e)
{
    if (H->size < H->cap) {
        int i = H->size++;
        H->h[i] = e;
        while (i > 0) {
            int p = (i - 1) / 2;
            if (!kv_gt(H->h[i], H->h[p])) break;
            kv t = H->h[i]; H->h[i] = H->h[p]; H->h[p] = t; i = p;
        }
    } else if (kv_gt(H->h[0], e)) {
        H->h[0] = e;
        int i = 0;
        for (;;) {
            int l = 2 * i + 1, r = l + 1, m = i;
            if (l < H->size && kv_gt(H->h[l], H->h[m])) m = l;
            if (r < H->size && kv_gt(H->h[r], H->h[m])) m = r;
            if (m == i) break;
            kv t = H->h[i]; H->h[i] = H->h[m]; H->h[m] = t; i = m;
        }
    }
}

static void kd_query_rec(const vto_kdtree* t, int64_t node, const float* q, int64_t self, kheap* H)
{
    const kd_node* nd = &t->nodes[node];
    if (nd->axis < 0) {
        for (int64_t i = nd->lo; i < nd->hi; ++i) {
            int64_t j = t->perm[i];
            if (j == self) continue;
            kv e = {dist2_f32(q, t->pts + 3 * j), j};
            kheap_push(H, e);
        }
        return;
    }
    double diff = (double)q[nd->axis] - nd->split;
    int64_t nearc = diff < 0 ? nd->left : nd->right, farc = diff < 0 ? nd->right : nd->left;
    kd_query_rec(t, nearc, q, self, H);
    /* every point on the far side has computed d2 >= fl(diff^2) (monotone rounding) */
    if (H->size < H->cap || diff * diff <= H->h[0].d2) kd_query_rec(t, farc, q, self, H);
}

static int kv_cmp(const void* a, const void* b)
{
    kv x = *(const kv*)a, y = *(const kv*)b;
    if (kv_gt(x, y)) return 1;
    if (kv_gt(y, x)) return -1;
    return 0;
}

/* k nearest of point `self` (excluded); writes up to k entries sorted by (d2, idx); returns count */
static int kd_knn(const vto_kdtree* t, int64_t self, int k, kv* out)
{
    kheap H = {out, 0, k};
    if (k > 0 && t->n > 0) kd_query_rec(t, 0, t->pts + 3 * self, self, &H);
    qsort(out, (size_t)H.size, sizeof(kv), kv_cmp);
    return H.size;
}

int vto_knn(const float* pts, int64_t n, const int64_t* queries, int64_t nq, int k,
            int32_t* nbr, double* d2, int nthreads)
{
    if (!pts || n < 0 || nq < 0 || k < 0 || (nq > 0 && !queries)) return VTO_ERR_ARG;
    vto_kdtree* t = vto_kdtree_build(pts, n);
    int status = VTO_OK;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        kv* buf = (kv*)malloc((size_t)(k > 0 ? k : 1) * sizeof(kv));
#pragma omp for schedule(dynamic, 256)
        for (int64_t q = 0; q < nq; ++q) {
            int64_t i = queries[q];
            if (i < 0 || i >= n) { status = VTO_ERR_ARG; continue; }
            int m = kd_knn(t, i, k, buf);
            for (int a = 0; a < k; ++a) {
                nbr[q * k + a] = a < m ? (int32_t)buf[a].idx : -1;
                if (d2) d2[q * k + a] = a < m ? buf[a].d2 : INFINITY;
            }
        }
        free(buf);
    }
    vto_kdtree_free(t);
    return status;
}

/* ------------------------------------------------------------------ */
/* convex polyhedron as a list of face polygons                        */
/* ------------------------------------------------------------------ */

#define MAXF 512   /* faces per polyhedron */
#define MAXFV 256  /* vertices per face    */

typedef struct {
    int32_t tag;   /* generator index (>= 0) or wall id -1..-6 */
    vec3 n;        /* plane n.x <= b in the local frame */
    double b;
    int nv;
    vec3 v[MAXFV];
} face_t;

typedef struct {
    int nf;
    face_t f[MAXF];
} poly_t;

/* per-thread scratch */
typedef struct {
    poly_t a, b;         /* current and next polyhedron */
    vec3 cap[MAXF * 2];  /* points of the cut */
    double ang[MAXF * 2];
    int order[MAXF * 2];
    vec3 tmp[MAXF * 2];
    kv* knn;             /* neighbour list buffer */
    int knn_cap;
    int64_t work_sign;   /* vertex-plane sign tests of the validating run */
    int64_t work_newv;   /* vertices created by cuts in the validating run */
    int64_t work_nbrs;   /* bisector planes tested in the validating run */
} scratch_t;

/* orthonormal in-plane basis (u, w) with u x w = n/|n| */
static void plane_basis(vec3 n, vec3* u, vec3* w)
{
    double nn = sqrt(vdot(n, n));
    vec3 nh = vscale(n, 1.0 / nn);
    vec3 e = fabs(nh.x) <= fabs(nh.y) && fabs(nh.x) <= fabs(nh.z) ? v3(1, 0, 0)
           : (fabs(nh.y) <= fabs(nh.z) ? v3(0, 1, 0) : v3(0, 0, 1));
    vec3 uu = vcross(nh, e);
    uu = vscale(uu, 1.0 / sqrt(vdot(uu, uu)));
    *u = uu;
    *w = vcross(nh, uu);
}

/* sort points of a planar convex polygon counter-clockwise seen from the tip of n */
static void sort_ccw(vec3* pts, int m, vec3 n, scratch_t* S)
{
    vec3 c = v3(0, 0, 0);
    for (int i = 0; i < m; ++i) c = vadd(c, pts[i]);
    c = vscale(c, 1.0 / m);
    vec3 u, w;
    plane_basis(n, &u, &w);
    for (int i = 0; i < m; ++i) {
        vec3 d = vsub(pts[i], c);
        S->ang[i] = atan2(vdot(d, w), vdot(d, u));
        S->order[i] = i;
    }
    /* insertion sort by angle (m is small) */
    for (int i = 1; i < m; ++i) {
        int o = S->order[i];
        int j = i - 1;
        while (j >= 0 && S->ang[S->order[j]] > S->ang[o]) { S->order[j + 1] = S->order[j]; --j; }
        S->order[j + 1] = o;
    }
    for (int i = 0; i < m; ++i) S->tmp[i] = pts[S->order[i]];
    memcpy(pts, S->tmp, (size_t)m * sizeof(vec3));
}

/* the domain box in the frame of generator p: faces with outward normals */
static void init_box(poly_t* P, vec3 lo, vec3 hi, scratch_t* S)
{
    /* wall ids: -1 x=lo, -2 x=hi, -3 y=lo, -4 y=hi, -5 z=lo, -6 z=hi */
    P->nf = 6;
    for (int w = 0; w < 6; ++w) {
        int axis = w / 2, upper = w % 2;
        face_t* F = &P->f[w];
        F->tag = -(w + 1);
        double nv[3] = {0, 0, 0};
        nv[axis] = upper ? 1.0 : -1.0;
        F->n = v3(nv[0], nv[1], nv[2]);
        double lov[3] = {lo.x, lo.y, lo.z}, hiv[3] = {hi.x, hi.y, hi.z};
        F->b = upper ? hiv[axis] : -lov[axis];
        int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
        F->nv = 4;
        for (int c = 0; c < 4; ++c) {
            double p[3];
            p[axis] = upper ? hiv[axis] : lov[axis];
            p[a1] = (c == 1 || c == 2) ? hiv[a1] : lov[a1];
            p[a2] = (c >= 2) ? hiv[a2] : lov[a2];
            F->v[c] = v3(p[0], p[1], p[2]);
        }
        sort_ccw(F->v, 4, F->n, S);
    }
}

static double side(vec3 n, double b, vec3 v) { return vdot(n, v) - b; }

/* canonical edge/plane intersection: always from the inside end to the outside end,
 * so the two faces sharing an edge produce the bit-identical point */
static vec3 cut_point(vec3 in, double s_in, vec3 out, double s_out)
{
    double t = s_in / (s_in - s_out);
    return vadd(in, vscale(vsub(out, in), t));
}

static int add_unique(vec3* set, int m, vec3 p)
{
    for (int i = 0; i < m; ++i) if (veq(set[i], p)) return m;
    set[m] = p;
    return m + 1;
}

/* clip P by the half-space n.x <= b (face tag `tag`) into Q: one step of the
 * cell-by-cell construction (Summary: the box is cut by the bisector of each
 * neighbour in turn). Returns 0 if nothing is cut (Q untouched), 1 if clipped
 * into Q, <0 on capacity error */
static int clip(const poly_t* P, poly_t* Q, vec3 n, double b, int32_t tag, scratch_t* S)
{
    int fv = 0;
    for (int f = 0; f < P->nf; ++f) fv += P->f[f].nv;
    S->work_sign += fv / 3;  /* each vertex of a simple polyhedron lies on 3 faces */
    S->work_nbrs += 1;
    int any_out = 0;
    for (int f = 0; f < P->nf && !any_out; ++f)
        for (int i = 0; i < P->f[f].nv; ++i)
            if (side(n, b, P->f[f].v[i]) > 0) { any_out = 1; break; }
    if (!any_out) return 0;

    int ncap = 0;
    Q->nf = 0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t* F = &P->f[f];
        face_t* G = &Q->f[Q->nf];
        int m = 0;
        for (int i = 0; i < F->nv; ++i) {
            vec3 a = F->v[i], c = F->v[(i + 1) % F->nv];
            double sa = side(n, b, a), sc = side(n, b, c);
            if (sa <= 0) {
                if (m >= MAXFV) return -1;
                G->v[m++] = a;
                if (sa == 0) { if (ncap >= MAXF * 2) return -1; ncap = add_unique(S->cap, ncap, a); }
            }
            if ((sa < 0 && sc > 0) || (sa > 0 && sc < 0)) {
                vec3 p = sa < 0 ? cut_point(a, sa, c, sc) : cut_point(c, sc, a, sa);
                if (m >= MAXFV) return -1;
                G->v[m++] = p;
                if (ncap >= MAXF * 2) return -1;
                int before = ncap;
                ncap = add_unique(S->cap, ncap, p);
                S->work_newv += ncap - before;
            }
        }
        /* drop repeated consecutive points (cyclic) */
        int k = 0;
        for (int i = 0; i < m; ++i)
            if (k == 0 || !veq(G->v[k - 1], G->v[i])) G->v[k++] = G->v[i];
        while (k > 1 && veq(G->v[0], G->v[k - 1])) --k;
        if (k >= 3) {
            G->nv = k; G->tag = F->tag; G->n = F->n; G->b = F->b;
            if (++Q->nf >= MAXF) return -1;
        }
    }
    if (ncap >= 3) {
        face_t* G = &Q->f[Q->nf];
        memcpy(G->v, S->cap, (size_t)ncap * sizeof(vec3));
        sort_ccw(G->v, ncap, n, S);
        G->nv = ncap; G->tag = tag; G->n = n; G->b = b;
        if (++Q->nf >= MAXF) return -1;
    }
    return 1;
}

static double max_r2(const poly_t* P)
{
    double r2 = 0;
    for (int f = 0; f < P->nf; ++f)
        for (int i = 0; i < P->f[f].nv; ++i) {
            double d = vdot(P->f[f].v[i], P->f[f].v[i]);
            if (d > r2) r2 = d;
        }
    return r2;
}

/* bisector of (p_i, p_j) in the local frame of p_i: n = p_j - p_i, b = |n|^2 / 2
 * (the points x with |x - p_i| = |x - p_j|; Statement of need: the Voronoi cell
 * is the set closer to p_i than to any other generator) */
static void bisector(const float* pi, const float* pj, vec3* n, double* b)
{
    *n = v3((double)pj[0] - (double)pi[0], (double)pj[1] - (double)pi[1], (double)pj[2] - (double)pi[2]);
    *b = 0.5 * vdot(*n, *n);
}

/* ------------------------------------------------------------------ */
/* periodic boxes                                                      */
/* ------------------------------------------------------------------ */

/* In a periodic box of periods L = hi - lo every generator p_j stands for all
 * its images p_j + t L, t integer. The cell of p_i is the set of points closer
 * to p_i than to any other image, p_i's own images included. The own images
 * at +-L_a e_a bound it by the cube [-L/2, L/2] around p_i (local frame); the
 * other own images only touch that cube at its edges and corners. So the cell
 * is that cube clipped by the bisectors of the images of the other
 * generators, its radius R is at most |L|/2, and only images closer than |L|
 * can cut it. With |L| <= 2 min_a L_a (required), an image with |t_a| >= 3 is
 * at least 2 L_a >= |L| away, so the shifts t in [-2, 2]^3 hold every image
 * that can cut. A shift is coded as (tx+2)*25 + (ty+2)*5 + (tz+2) (62 = none)
 * and a face of a periodic cell is tagged j*128 + code (the cube's faces
 * with j = i and the shift of the own image across them). */
#define IMG_NONE 62
#define IMG_CODES 125

static int img_code(int tx, int ty, int tz) { return (tx + 2) * 25 + (ty + 2) * 5 + (tz + 2); }
static void img_shift(int code, int t[3]) { t[0] = code / 25 - 2; t[1] = (code / 5) % 5 - 2; t[2] = code % 5 - 2; }

/* offset of image (j, code) from p_i: per coordinate ((x_j - x_i) + t L) in
 * double; the kNN key is its squared length ((dx*dx + dy*dy) + dz*dz) */
static vec3 image_offset(const float* pi, const float* pj, int code, vec3 L)
{
    int t[3];
    img_shift(code, t);
    return v3(((double)pj[0] - (double)pi[0]) + (double)t[0] * L.x,
              ((double)pj[1] - (double)pi[1]) + (double)t[1] * L.y,
              ((double)pj[2] - (double)pi[2]) + (double)t[2] * L.z);
}

/* the cube [-L/2, L/2] around generator i, faces tagged with i's own images */
static void init_cube(poly_t* P, int64_t i, vec3 L, scratch_t* S)
{
    vec3 h = vscale(L, 0.5);
    init_box(P, vscale(h, -1.0), h, S);
    for (int f = 0; f < P->nf; ++f) {
        int w = -P->f[f].tag - 1, axis = w / 2, s = (w % 2) ? 1 : -1;
        P->f[f].tag = (int32_t)(i * 128 + img_code(axis == 0 ? s : 0, axis == 1 ? s : 0, axis == 2 ? s : 0));
    }
}

/* kd-tree over the images that lie within `margin` of the box (shifts in
 * {-1, 0, 1}^3): it holds every image closer than `margin` to any point of
 * the box. Image coordinates only partition the tree; keys are always the
 * image_offset expression above. */
typedef struct {
    const float* pts;
    vec3 L;
    int64_t m;
    double* X;      /* [3m] image coordinates */
    int64_t* id;    /* [m] j * 128 + code */
    int64_t* perm;
    kd_node* nodes;
    int64_t n_nodes, cap_nodes;
} img_tree;

static int img_less(const img_tree* t, int64_t a, int64_t b, int axis)
{
    double ca = t->X[3 * a + axis], cb = t->X[3 * b + axis];
    return ca < cb || (ca == cb && t->id[a] < t->id[b]);
}

static void img_select(img_tree* t, int64_t lo, int64_t hi, int64_t m, int axis)
{
    int64_t* p = t->perm;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t tmp = p[mid]; p[mid] = p[hi - 1]; p[hi - 1] = tmp;
        int64_t pv = p[hi - 1], store = lo;
        for (int64_t i = lo; i < hi - 1; ++i)
            if (img_less(t, p[i], pv, axis)) { tmp = p[i]; p[i] = p[store]; p[store] = tmp; ++store; }
        tmp = p[store]; p[store] = p[hi - 1]; p[hi - 1] = tmp;
        if (store == m) return;
        if (m < store) hi = store; else lo = store + 1;
    }
}

static int64_t img_build_rec(img_tree* t, int64_t lo, int64_t hi)
{
    if (t->n_nodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes * 2 + 16;
        t->nodes = (kd_node*)realloc(t->nodes, (size_t)t->cap_nodes * sizeof(kd_node));
    }
    int64_t id = t->n_nodes++;
    t->nodes[id].lo = lo; t->nodes[id].hi = hi;
    t->nodes[id].axis = -1; t->nodes[id].left = t->nodes[id].right = -1;
    if (hi - lo <= KD_LEAF) return id;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = lo; i < hi; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = t->X[3 * t->perm[i] + a];
            if (c < mn[a]) mn[a] = c;
            if (c > mx[a]) mx[a] = c;
        }
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (mx[a] - mn[a] > mx[axis] - mn[axis]) axis = a;
    int64_t m = lo + (hi - lo) / 2;
    img_select(t, lo, hi, m, axis);
    t->nodes[id].axis = axis;
    t->nodes[id].split = t->X[3 * t->perm[m] + axis];
    int64_t l = img_build_rec(t, lo, m);
    int64_t r = img_build_rec(t, m, hi);
    t->nodes[id].left = l; t->nodes[id].right = r;
    return id;
}

static img_tree* img_tree_build(const float* pts, int64_t n, vec3 lo, vec3 L, double margin)
{
    img_tree* t = (img_tree*)calloc(1, sizeof(img_tree));
    t->pts = pts; t->L = L;
    t->X = (double*)malloc((size_t)(27 * n + 1) * 3 * sizeof(double));
    t->id = (int64_t*)malloc((size_t)(27 * n + 1) * sizeof(int64_t));
    double lov[3] = {lo.x, lo.y, lo.z}, Lv[3] = {L.x, L.y, L.z};
    int64_t m = 0;
    for (int64_t j = 0; j < n; ++j)
        for (int tx = -1; tx <= 1; ++tx)
            for (int ty = -1; ty <= 1; ++ty)
                for (int tz = -1; tz <= 1; ++tz) {
                    int tv[3] = {tx, ty, tz}, keep = 1;
                    double x[3];
                    for (int a = 0; a < 3; ++a) {
                        x[a] = (double)pts[3 * j + a] + (double)tv[a] * Lv[a];
                        if (!(x[a] >= lov[a] - margin && x[a] < lov[a] + Lv[a] + margin)) keep = 0;
                    }
                    if (!keep) continue;
                    t->X[3 * m] = x[0]; t->X[3 * m + 1] = x[1]; t->X[3 * m + 2] = x[2];
                    t->id[m] = j * 128 + img_code(tx, ty, tz);
                    ++m;
                }
    t->m = m;
    t->perm = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) t->perm[i] = i;
    if (m > 0) img_build_rec(t, 0, m);
    return t;
}

static void img_tree_free(img_tree* t)
{
    if (!t) return;
    free(t->X); free(t->id); free(t->perm); free(t->nodes); free(t);
}

static void img_query_rec(const img_tree* t, int64_t node, int64_t self, const double* q, kheap* H)
{
    const kd_node* nd = &t->nodes[node];
    if (nd->axis < 0) {
        for (int64_t r = nd->lo; r < nd->hi; ++r) {
            int64_t id = t->id[t->perm[r]];
            int64_t j = id >> 7;
            if (j == self) continue;
            vec3 o = image_offset(t->pts + 3 * self, t->pts + 3 * j, (int)(id & 127), t->L);
            kv e = {vdot(o, o), id};
            kheap_push(H, e);
        }
        return;
    }
    double diff = q[nd->axis] - nd->split;
    int64_t nearc = diff < 0 ? nd->left : nd->right, farc = diff < 0 ? nd->right : nd->left;
    img_query_rec(t, nearc, self, q, H);
    /* a far-side image is at least |diff| away; keys carry ~1e-15 relative rounding */
    if (H->size < H->cap || diff * diff <= H->h[0].d2 * (1.0 + 1e-9)) img_query_rec(t, farc, self, q, H);
}

/* the k nearest images of generator `self` in the tree, sorted by (key, j, code) */
static int img_knn(const img_tree* t, int64_t self, int k, kv* out)
{
    kheap H = {out, 0, k};
    double q[3] = {t->pts[3 * self], t->pts[3 * self + 1], t->pts[3 * self + 2]};
    if (k > 0 && t->m > 0) img_query_rec(t, 0, self, q, &H);
    qsort(out, (size_t)H.size, sizeof(kv), kv_cmp);
    return H.size;
}

/* every image (j != self, t in [-2, 2]^3) sorted by (key, j, code); returns a
 * malloc'd array of *m entries */
static kv* img_all(const float* pts, int64_t n, vec3 L, int64_t self, int64_t* m)
{
    int64_t cnt = (n - 1) * IMG_CODES, w = 0;
    kv* a = (kv*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(kv));
    for (int64_t j = 0; j < n; ++j) {
        if (j == self) continue;
        for (int c = 0; c < IMG_CODES; ++c) {
            vec3 o = image_offset(pts + 3 * self, pts + 3 * j, c, L);
            kv e = {vdot(o, o), j * 128 + c};
            a[w++] = e;
        }
    }
    qsort(a, (size_t)w, sizeof(kv), kv_cmp);
    *m = w;
    return a;
}

static double min3(vec3 a) { return fmin(a.x, fmin(a.y, a.z)); }

/* periodic box accepted: positive periods with |L|^2 <= 4 min L_a^2, n < 2^24 */
static int periodic_ok(vec3 L, int64_t n)
{
    double lm = min3(L);
    return lm > 0 && vdot(L, L) <= 4.0 * lm * lm && n < ((int64_t)1 << 24);
}

/* ------------------------------------------------------------------ */
/* vertex positions from their planes                                  */
/* ------------------------------------------------------------------ */

#define SNAP_INC 8  /* faces remembered per vertex */

/* solve the 3x3 system n_r . x = b_r by Gaussian elimination with partial
 * pivoting; returns 0 if a pivot vanishes */
static int solve_planes(const vec3* n, const double* b, vec3* x)
{
    double A[3][4] = {{n[0].x, n[0].y, n[0].z, b[0]}, {n[1].x, n[1].y, n[1].z, b[1]}, {n[2].x, n[2].y, n[2].z, b[2]}};
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0) return 0;
        if (piv != c)
            for (int k = 0; k < 4; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        for (int r = c + 1; r < 3; ++r) {
            double f = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= f * A[c][k];
        }
    }
    double z = A[2][3] / A[2][2];
    double y = (A[1][3] - A[1][2] * z) / A[1][1];
    double xx = (A[0][3] - A[0][1] * y - A[0][2] * z) / A[0][0];
    *x = v3(xx, y, z);
    return 1;
}

/* Every vertex of the final cell is the common point of the planes of the
 * faces that meet there (the cell is the box cut by bisector planes). The
 * clipper reaches it by interpolating along edges, whose rounding scales with
 * the length of the edge it cut -- up to the size of the box, far above the
 * size of a small cell. Each vertex (vertices closer than 1e-12 V^(1/3) are
 * one) is therefore recomputed from the triple of its face planes with the
 * largest |det| of unit normals, when that is at least 1e-6; otherwise the
 * interpolated position stays. */
static void snap_vertices(poly_t* P, vec3* uniq, int* vid, int* inc, int* ninc)
{
    double vol = 0;
    for (int f = 0; f < P->nf; ++f)
        for (int i = 1; i + 1 < P->f[f].nv; ++i) vol += vdet(P->f[f].v[0], P->f[f].v[i], P->f[f].v[i + 1]) / 6.0;
    double tol = 1e-12 * cbrt(fabs(vol));
    int nu = 0, pos = 0;
    for (int f = 0; f < P->nf; ++f)
        for (int i = 0; i < P->f[f].nv; ++i) {
            vec3 v = P->f[f].v[i];
            int id = -1;
            for (int u = 0; u < nu && id < 0; ++u)
                if (fabs(uniq[u].x - v.x) <= tol && fabs(uniq[u].y - v.y) <= tol && fabs(uniq[u].z - v.z) <= tol)
                    id = u;
            if (id < 0) { uniq[nu] = v; ninc[nu] = 0; id = nu++; }
            vid[pos++] = id;
            int seen = 0;
            for (int t = 0; t < ninc[id] && t < SNAP_INC; ++t) seen |= inc[id * SNAP_INC + t] == f;
            if (!seen && ninc[id] < SNAP_INC) inc[id * SNAP_INC + ninc[id]++] = f;
        }
    for (int u = 0; u < nu; ++u) {
        int m = ninc[u];
        if (m < 3) continue;
        double best = 0;
        int ba = -1, bb = -1, bc = -1;
        vec3 h[SNAP_INC];
        for (int t = 0; t < m; ++t) {
            vec3 nn = P->f[inc[u * SNAP_INC + t]].n;
            h[t] = vscale(nn, 1.0 / sqrt(vdot(nn, nn)));
        }
        for (int a = 0; a < m; ++a)
            for (int b = a + 1; b < m; ++b)
                for (int c = b + 1; c < m; ++c) {
                    double d = fabs(vdet(h[a], h[b], h[c]));
                    if (d > best) { best = d; ba = a; bb = b; bc = c; }
                }
        if (best < 1e-6) continue;
        const face_t* Fa = &P->f[inc[u * SNAP_INC + ba]];
        const face_t* Fb = &P->f[inc[u * SNAP_INC + bb]];
        const face_t* Fc = &P->f[inc[u * SNAP_INC + bc]];
        vec3 nrm[3] = {Fa->n, Fb->n, Fc->n};
        double rhs[3] = {Fa->b, Fb->b, Fc->b};
        vec3 x;
        if (solve_planes(nrm, rhs, &x)) uniq[u] = x;
    }
    pos = 0;
    for (int f = 0; f < P->nf; ++f)
        for (int i = 0; i < P->f[f].nv; ++i) P->f[f].v[i] = uniq[vid[pos++]];
}

/* ------------------------------------------------------------------ */
/* per-cell measures                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    double vol, cen[3], m2;
    int nfaces, nvert, nedge;   /* topology after merging near-coincident vertices */
} cell_meas;

/* Volume, first and second moment by a tetrahedron fan from the generator
 * (the local origin, inside its own cell); face area and centroid by a
 * triangle fan from the face's first vertex. The paper's library returns
 * several per-cell outputs and names the neighbour lists among them
 * (Features); these moments are the ones this implementation returns beside
 * the neighbours (a Lloyd step needs volume and centroid).
 *
 * Topology: exact FP64 clipping at degenerate inputs (lattices) can leave
 * vertices a few ulps apart and zero-area sliver faces. For the reported
 * topology, vertices closer than 1e-12 V^(1/3) (max-norm) are merged, each
 * face loop is cleaned of repeated points, and faces left with fewer than 3
 * distinct vertices are dropped (lsize[f] = 0). loop[] receives the cleaned
 * loops back to back as indices into uniq[]. */
static void measure(const poly_t* P, vec3 pi, cell_meas* M, double* farea, vec3* fcen,
                    vec3* uniq, int* loop, int* lsize, char* used)
{
    double vol = 0, m2 = 0;
    vec3 mom = v3(0, 0, 0);
    for (int f = 0; f < P->nf; ++f) {
        const face_t* F = &P->f[f];
        vec3 nh = vscale(F->n, 1.0 / sqrt(vdot(F->n, F->n)));
        double area = 0;
        vec3 amom = v3(0, 0, 0);
        for (int i = 1; i + 1 < F->nv; ++i) {
            vec3 a = F->v[0], b = F->v[i], c = F->v[i + 1];
            double dv = vdet(a, b, c) / 6.0;
            vec3 s = vadd(vadd(a, b), c);
            vol += dv;
            mom = vadd(mom, vscale(s, dv / 4.0));
            m2 += dv / 20.0 * (vdot(a, a) + vdot(b, b) + vdot(c, c) + vdot(s, s));
            double ta = 0.5 * vdot(vcross(vsub(b, a), vsub(c, a)), nh);
            area += ta;
            amom = vadd(amom, vscale(s, ta / 3.0));
        }
        farea[f] = area;
        fcen[f] = area != 0 ? vadd(pi, vscale(amom, 1.0 / area)) : pi;
    }
    M->vol = vol;
    M->cen[0] = pi.x + mom.x / vol;
    M->cen[1] = pi.y + mom.y / vol;
    M->cen[2] = pi.z + mom.z / vol;
    M->m2 = m2;

    double tol = 1e-12 * cbrt(vol);
    int nu = 0, pos = 0, nedge2 = 0, nfaces = 0;
    for (int f = 0; f < P->nf; ++f) {
        const face_t* F = &P->f[f];
        int start = pos;
        for (int i = 0; i < F->nv; ++i) {
            vec3 v = F->v[i];
            int id = -1;
            for (int u = 0; u < nu && id < 0; ++u)
                if (fabs(uniq[u].x - v.x) <= tol && fabs(uniq[u].y - v.y) <= tol && fabs(uniq[u].z - v.z) <= tol)
                    id = u;
            if (id < 0) { uniq[nu] = v; used[nu] = 0; id = nu++; }
            if (pos == start || loop[pos - 1] != id) loop[pos++] = id;
        }
        while (pos - start > 1 && loop[pos - 1] == loop[start]) --pos;
        if (pos - start >= 3) {
            lsize[f] = pos - start;
            nedge2 += lsize[f];
            ++nfaces;
            for (int i = start; i < pos; ++i) used[loop[i]] = 1;
        } else {
            lsize[f] = 0;
            pos = start;
        }
    }
    int nv = 0;
    for (int u = 0; u < nu; ++u) nv += used[u];
    M->nfaces = nfaces;
    M->nedge = nedge2 / 2;
    M->nvert = nv;
}

/* ------------------------------------------------------------------ */
/* one cell                                                            */
/* ------------------------------------------------------------------ */

/* Computes the cell of generator i into *out_poly (a pointer into S).
 * mode VTO_MODE_SECURITY: kNN + security radius with k doubling (Summary: the
 * neighbours nearest first, stopping once the security radius shows that no
 * farther generator can cut the cell, and a larger k when the list runs out).
 * mode VTO_MODE_BRUTE: every other generator, in index order (order == NULL)
 *   or in the order given by `order` (a permutation of 0..n-1), no stop test.
 * Returns status; *k_used gets the final k (n-1 for brute force). */
static int one_cell(const float* pts, int64_t n, vec3 lo, vec3 hi, const vto_kdtree* T,
                    int64_t i, int k0, int mode, const int64_t* order,
                    scratch_t* S, poly_t** out_poly, int* k_used, int* n_clips)
{
    const float* pi = pts + 3 * i;
    vec3 p = v3(pi[0], pi[1], pi[2]);
    vec3 llo = vsub(lo, p), lhi = vsub(hi, p);
    *n_clips = 0;

    if (mode != VTO_MODE_SECURITY) {
        S->work_sign = S->work_newv = S->work_nbrs = 0;
        poly_t *cur = &S->a, *nxt = &S->b;
        init_box(cur, llo, lhi, S);
        for (int64_t t = 0; t < n; ++t) {
            int64_t j = order ? order[t] : t;
            if (j == i) continue;
            vec3 nn; double b;
            bisector(pi, pts + 3 * j, &nn, &b);
            if (b == 0) return VTO_ERR_DUPLICATE;
            int r = clip(cur, nxt, nn, b, (int32_t)j, S);
            if (r < 0) return VTO_ERR_CAPACITY;
            if (r == 1) { poly_t* tmp = cur; cur = nxt; nxt = tmp; ++*n_clips; }
        }
        *out_poly = cur;
        *k_used = (int)(n - 1);
        return VTO_OK;
    }

    int64_t k = k0 > 0 ? k0 : 1;
    for (;;) {
        int64_t keff = k < n - 1 ? k : n - 1;
        if (keff > S->knn_cap) {
            S->knn_cap = (int)keff;
            S->knn = (kv*)realloc(S->knn, (size_t)keff * sizeof(kv));
        }
        int m = kd_knn(T, i, (int)keff, S->knn);
        poly_t *cur = &S->a, *nxt = &S->b;
        init_box(cur, llo, lhi, S);
        int valid = 0;
        *n_clips = 0;
        S->work_sign = S->work_newv = S->work_nbrs = 0;
        for (int a = 0; a < m; ++a) {
            if (S->knn[a].d2 == 0) return VTO_ERR_DUPLICATE;
            if (4.0 * max_r2(cur) <= S->knn[a].d2) { valid = 1; break; }
            vec3 nn; double b;
            bisector(pi, pts + 3 * S->knn[a].idx, &nn, &b);
            int r = clip(cur, nxt, nn, b, (int32_t)S->knn[a].idx, S);
            if (r < 0) return VTO_ERR_CAPACITY;
            if (r == 1) { poly_t* tmp = cur; cur = nxt; nxt = tmp; ++*n_clips; }
        }
        if (!valid) {
            if (m == n - 1) valid = 1;                                   /* every generator used */
            else if (m > 0 && 4.0 * max_r2(cur) <= S->knn[m - 1].d2) valid = 1;
        }
        if (valid) { *out_poly = cur; *k_used = (int)keff; return VTO_OK; }
        k *= 2;
    }
}

/* The periodic cell of generator i (see "periodic boxes"): the cube around
 * p_i clipped by the images of the other generators. Security mode takes the
 * images nearest first from the margin tree with the security-radius stop and
 * k doubling, as one_cell does; the tree holds every image closer than lim^(1/2),
 * so a cell that is not final before its list reaches that distance (or
 * that runs out of images) is finished from the sorted list of all images.
 * Brute mode clips by every image of every other generator, j in index (or
 * `order`) order, shift codes ascending. */
static int one_cell_periodic(const float* pts, int64_t n, vec3 L, const img_tree* T, double lim,
                             int64_t i, int k0, int mode, const int64_t* order,
                             scratch_t* S, poly_t** out_poly, int* k_used, int* n_clips)
{
    const float* pi = pts + 3 * i;
    poly_t *cur = &S->a, *nxt = &S->b;
    *n_clips = 0;
    S->work_sign = S->work_newv = S->work_nbrs = 0;
    if (mode != VTO_MODE_SECURITY) {
        init_cube(cur, i, L, S);
        for (int64_t t = 0; t < n; ++t) {
            int64_t j = order ? order[t] : t;
            if (j == i) continue;
            for (int c = 0; c < IMG_CODES; ++c) {
                vec3 nn = image_offset(pi, pts + 3 * j, c, L);
                double b = 0.5 * vdot(nn, nn);
                if (b == 0) return VTO_ERR_DUPLICATE;
                int r = clip(cur, nxt, nn, b, (int32_t)(j * 128 + c), S);
                if (r < 0) return VTO_ERR_CAPACITY;
                if (r == 1) { poly_t* tmp = cur; cur = nxt; nxt = tmp; ++*n_clips; }
            }
        }
        *out_poly = cur;
        *k_used = (int)(n - 1);
        return VTO_OK;
    }

    int64_t k = k0 > 0 ? k0 : 1;
    int all = 0;
    for (;;) {
        if (k > S->knn_cap) {
            S->knn_cap = (int)k;
            S->knn = (kv*)realloc(S->knn, (size_t)k * sizeof(kv));
        }
        int m = img_knn(T, i, (int)k, S->knn);
        cur = &S->a; nxt = &S->b;
        init_cube(cur, i, L, S);
        int valid = 0;
        *n_clips = 0;
        S->work_sign = S->work_newv = S->work_nbrs = 0;
        for (int a = 0; a < m; ++a) {
            if (S->knn[a].d2 == 0) return VTO_ERR_DUPLICATE;
            if (4.0 * max_r2(cur) <= S->knn[a].d2) { valid = 1; break; }
            if (S->knn[a].d2 >= lim) { all = 1; break; }
            vec3 nn = image_offset(pi, pts + 3 * (S->knn[a].idx >> 7), (int)(S->knn[a].idx & 127), L);
            int r = clip(cur, nxt, nn, 0.5 * vdot(nn, nn), (int32_t)S->knn[a].idx, S);
            if (r < 0) return VTO_ERR_CAPACITY;
            if (r == 1) { poly_t* tmp = cur; cur = nxt; nxt = tmp; ++*n_clips; }
        }
        if (!valid && !all) {
            if (m < k) all = 1;
            else if (4.0 * max_r2(cur) <= S->knn[m - 1].d2) valid = 1;
        }
        if (valid) { *out_poly = cur; *k_used = (int)k; return VTO_OK; }
        if (all) break;
        k *= 2;
    }

    int64_t m = 0;
    kv* list = img_all(pts, n, L, i, &m);
    cur = &S->a; nxt = &S->b;
    init_cube(cur, i, L, S);
    *n_clips = 0;
    S->work_sign = S->work_newv = S->work_nbrs = 0;
    int st = VTO_OK;
    for (int64_t a = 0; a < m; ++a) {
        if (list[a].d2 == 0) { st = VTO_ERR_DUPLICATE; break; }
        if (4.0 * max_r2(cur) <= list[a].d2) break;
        vec3 nn = image_offset(pi, pts + 3 * (list[a].idx >> 7), (int)(list[a].idx & 127), L);
        int r = clip(cur, nxt, nn, 0.5 * vdot(nn, nn), (int32_t)list[a].idx, S);
        if (r < 0) { st = VTO_ERR_CAPACITY; break; }
        if (r == 1) { poly_t* tmp = cur; cur = nxt; nxt = tmp; ++*n_clips; }
    }
    free(list);
    *out_poly = cur;
    *k_used = m < INT32_MAX ? (int)m : INT32_MAX;
    return st;
}

/* ------------------------------------------------------------------ */
/* driver                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    int status;
    int nf, nv;
    int32_t* tag;     /* [nf] */
    double* area;     /* [nf] */
    double* fcen;     /* [nf*3] */
    double* fnrm;     /* [nf*4] plane n (global frame: same vector), b (local) */
    int32_t* fsize;   /* [nf] */
    double* fvtx;     /* [sum fsize * 3] global coordinates */
    int32_t* nbr; int nnbr;
    cell_meas M;
    int k_used, n_clips;
    int64_t work_sign, work_newv, work_nbrs;
} cell_rec;

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static int tess_impl(const float* pts, int64_t n, const float lo_f[3], const float hi_f[3],
                     int k0, int mode, const int64_t* order,
                     const int64_t* cells, int64_t n_cells, int want_geometry, int nthreads, int periodic,
                     vto_result** result)
{
    if (!result || !pts || n < 0 || !lo_f || !hi_f) return VTO_ERR_ARG;
    *result = NULL;
    vec3 lo = v3(lo_f[0], lo_f[1], lo_f[2]), hi = v3(hi_f[0], hi_f[1], hi_f[2]);
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float c = pts[3 * i + a];
            if (!(c >= lo_f[a] && c < hi_f[a])) return VTO_ERR_ARG;
        }
    vec3 L = v3((double)hi_f[0] - (double)lo_f[0], (double)hi_f[1] - (double)lo_f[1],
                (double)hi_f[2] - (double)lo_f[2]);
    if (periodic && !periodic_ok(L, n)) return VTO_ERR_ARG;
    int64_t nc = cells ? n_cells : n;
    vto_result* R = (vto_result*)calloc(1, sizeof(vto_result));
    R->n_cells = nc;
    R->vol = (double*)calloc((size_t)nc + 1, sizeof(double));
    R->cen = (double*)calloc((size_t)nc * 3 + 1, sizeof(double));
    R->m2 = (double*)calloc((size_t)nc + 1, sizeof(double));
    R->nbr_off = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    R->k_used = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
    R->n_clips = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
    R->euler = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
    R->nvert = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
    R->face_off = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    R->periodic = periodic;
    R->work_sign = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    R->work_newv = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    R->work_nbrs = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    cell_rec* recs = (cell_rec*)calloc((size_t)nc + 1, sizeof(cell_rec));
    vto_kdtree* T = mode == VTO_MODE_SECURITY && !periodic ? vto_kdtree_build(pts, n) : NULL;
    /* periodic: the tree holds every image within half the shortest period of the box */
    img_tree* TP = mode == VTO_MODE_SECURITY && periodic ? img_tree_build(pts, n, lo, L, 0.5 * min3(L)) : NULL;
    const double lim = 0.25 * min3(L) * min3(L) * (1.0 - 1e-9);
    int status = VTO_OK;

#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        scratch_t* S = (scratch_t*)calloc(1, sizeof(scratch_t));
        double* farea = (double*)malloc(MAXF * sizeof(double));
        vec3* fcen = (vec3*)malloc(MAXF * sizeof(vec3));
        vec3* uniq = (vec3*)malloc((size_t)MAXF * MAXFV * sizeof(vec3));
        int* loop = (int*)malloc((size_t)MAXF * MAXFV * sizeof(int));
        int* lsize = (int*)malloc((size_t)MAXF * sizeof(int));
        char* used = (char*)malloc((size_t)MAXF * MAXFV);
        int* sinc = (int*)malloc((size_t)MAXF * MAXFV * SNAP_INC * sizeof(int));
        int* sninc = (int*)malloc((size_t)MAXF * MAXFV * sizeof(int));
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < nc; ++c) {
            int64_t i = cells ? cells[c] : c;
            cell_rec* rc = &recs[c];
            if (i < 0 || i >= n) { rc->status = VTO_ERR_ARG; continue; }
            poly_t* P = NULL;
            rc->status = periodic
                ? one_cell_periodic(pts, n, L, TP, lim, i, k0, mode, order, S, &P, &rc->k_used, &rc->n_clips)
                : one_cell(pts, n, lo, hi, T, i, k0, mode, order, S, &P, &rc->k_used, &rc->n_clips);
            rc->work_sign = S->work_sign;
            rc->work_newv = S->work_newv;
            rc->work_nbrs = S->work_nbrs;
            if (rc->status != VTO_OK) continue;
            vec3 p = v3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
            snap_vertices(P, uniq, loop, sinc, sninc);
            measure(P, p, &rc->M, farea, fcen, uniq, loop, lsize, used);
            double tau = 1e-12 * pow(rc->M.vol, 2.0 / 3.0);
            int nf = rc->M.nfaces;
            rc->nf = nf;
            rc->tag = (int32_t*)malloc((size_t)nf * sizeof(int32_t) + 4);
            rc->area = (double*)malloc((size_t)nf * sizeof(double) + 8);
            rc->fcen = (double*)malloc((size_t)nf * 3 * sizeof(double) + 8);
            rc->fnrm = (double*)malloc((size_t)nf * 4 * sizeof(double) + 8);
            rc->fsize = (int32_t*)malloc((size_t)nf * sizeof(int32_t) + 4);
            rc->nbr = (int32_t*)malloc((size_t)nf * sizeof(int32_t) + 4);
            int nv = 0;
            for (int f = 0; f < P->nf; ++f) nv += lsize[f];
            rc->nv = nv;
            rc->fvtx = want_geometry ? (double*)malloc((size_t)nv * 3 * sizeof(double) + 8) : NULL;
            int w = 0, g = 0, lp = 0;
            rc->nnbr = 0;
            for (int f = 0; f < P->nf; ++f) {
                if (lsize[f] == 0) continue;
                const face_t* F = &P->f[f];
                rc->tag[g] = F->tag;
                rc->area[g] = farea[f];
                rc->fcen[3 * g] = fcen[f].x; rc->fcen[3 * g + 1] = fcen[f].y; rc->fcen[3 * g + 2] = fcen[f].z;
                rc->fnrm[4 * g] = F->n.x; rc->fnrm[4 * g + 1] = F->n.y; rc->fnrm[4 * g + 2] = F->n.z;
                rc->fnrm[4 * g + 3] = F->b;
                rc->fsize[g] = lsize[f];
                if (rc->fvtx)
                    for (int v = 0; v < lsize[f]; ++v, ++w) {
                        vec3 u = uniq[loop[lp + v]];
                        rc->fvtx[3 * w] = p.x + u.x;
                        rc->fvtx[3 * w + 1] = p.y + u.y;
                        rc->fvtx[3 * w + 2] = p.z + u.z;
                    }
                lp += lsize[f];
                if (F->tag >= 0 && farea[f] > tau) rc->nbr[rc->nnbr++] = periodic ? F->tag >> 7 : F->tag;
                ++g;
            }
            qsort(rc->nbr, (size_t)rc->nnbr, sizeof(int32_t), cmp_i32);
        }
        free(S->knn); free(S); free(farea); free(fcen); free(uniq); free(loop); free(lsize); free(used);
        free(sinc); free(sninc);
    }

    /* gather into flat arrays */
    int64_t tot_nbr = 0, tot_f = 0, tot_v = 0;
    for (int64_t c = 0; c < nc; ++c) {
        if (recs[c].status != VTO_OK && status == VTO_OK) status = recs[c].status;
        tot_nbr += recs[c].nnbr; tot_f += recs[c].nf; tot_v += recs[c].nv;
    }
    R->nbr = (int32_t*)malloc((size_t)tot_nbr * sizeof(int32_t) + 4);
    R->face_tag = (int32_t*)malloc((size_t)tot_f * sizeof(int32_t) + 4);
    R->face_area = (double*)malloc((size_t)tot_f * sizeof(double) + 8);
    R->face_cen = (double*)malloc((size_t)tot_f * 3 * sizeof(double) + 8);
    R->face_plane = (double*)malloc((size_t)tot_f * 4 * sizeof(double) + 8);
    R->face_size = (int32_t*)malloc((size_t)tot_f * sizeof(int32_t) + 4);
    R->face_img = (int32_t*)malloc((size_t)tot_f * sizeof(int32_t) + 4);
    R->face_vtx = want_geometry ? (double*)malloc((size_t)tot_v * 3 * sizeof(double) + 8) : NULL;
    R->n_nbr = tot_nbr; R->n_faces = tot_f; R->n_face_vtx = tot_v;
    int64_t on = 0, of = 0, ov = 0;
    for (int64_t c = 0; c < nc; ++c) {
        cell_rec* rc = &recs[c];
        R->nbr_off[c] = on; R->face_off[c] = of;
        if (rc->status == VTO_OK) {
            R->vol[c] = rc->M.vol;
            R->cen[3 * c] = rc->M.cen[0]; R->cen[3 * c + 1] = rc->M.cen[1]; R->cen[3 * c + 2] = rc->M.cen[2];
            R->m2[c] = rc->M.m2;
            R->euler[c] = rc->M.nvert - rc->M.nedge + rc->M.nfaces;
            R->nvert[c] = rc->M.nvert;
            memcpy(R->nbr + on, rc->nbr, (size_t)rc->nnbr * sizeof(int32_t));
            for (int g = 0; g < rc->nf; ++g) {
                R->face_tag[of + g] = periodic ? rc->tag[g] >> 7 : rc->tag[g];
                R->face_img[of + g] = periodic ? rc->tag[g] & 127 : IMG_NONE;
            }
            memcpy(R->face_area + of, rc->area, (size_t)rc->nf * sizeof(double));
            memcpy(R->face_cen + 3 * of, rc->fcen, (size_t)rc->nf * 3 * sizeof(double));
            memcpy(R->face_plane + 4 * of, rc->fnrm, (size_t)rc->nf * 4 * sizeof(double));
            memcpy(R->face_size + of, rc->fsize, (size_t)rc->nf * sizeof(int32_t));
            if (R->face_vtx) memcpy(R->face_vtx + 3 * ov, rc->fvtx, (size_t)rc->nv * 3 * sizeof(double));
            on += rc->nnbr; of += rc->nf; ov += rc->nv;
        }
        R->k_used[c] = rc->k_used;
        R->n_clips[c] = rc->n_clips;
        R->work_sign[c] = rc->work_sign;
        R->work_newv[c] = rc->work_newv;
        R->work_nbrs[c] = rc->work_nbrs;
        free(rc->tag); free(rc->area); free(rc->fcen); free(rc->fnrm); free(rc->fsize);
        free(rc->fvtx); free(rc->nbr);
    }
    R->nbr_off[nc] = on; R->face_off[nc] = of;
    free(recs);
    vto_kdtree_free(T);
    img_tree_free(TP);
    R->status = status;
    *result = R;
    return status;
}

void vto_result_free(vto_result* R)
{
    if (!R) return;
    free(R->vol); free(R->cen); free(R->m2); free(R->nbr_off); free(R->nbr);
    free(R->k_used); free(R->n_clips); free(R->euler); free(R->nvert);
    free(R->face_off); free(R->face_tag); free(R->face_area); free(R->face_cen);
    free(R->face_plane); free(R->face_size); free(R->face_vtx);
    free(R->work_sign); free(R->work_newv); free(R->work_nbrs); free(R->face_img);
    free(R);
}

int vto_tessellate(const float* pts, int64_t n, const float lo_f[3], const float hi_f[3],
                   int k0, int mode, const int64_t* order,
                   const int64_t* cells, int64_t n_cells, int want_geometry, int nthreads,
                   vto_result** result)
{
    return tess_impl(pts, n, lo_f, hi_f, k0, mode, order, cells, n_cells, want_geometry, nthreads, 0, result);
}

int vto_tessellate_periodic(const float* pts, int64_t n, const float lo_f[3], const float hi_f[3],
                            int k0, int mode, const int64_t* order,
                            const int64_t* cells, int64_t n_cells, int want_geometry, int nthreads,
                            vto_result** result)
{
    return tess_impl(pts, n, lo_f, hi_f, k0, mode, order, cells, n_cells, want_geometry, nthreads, 1, result);
}

int vto_knn_periodic(const float* pts, int64_t n, const float lo_f[3], const float hi_f[3],
                     const int64_t* queries, int64_t nq, int k, int32_t* nbr, int32_t* img, double* d2,
                     int nthreads)
{
    if (!pts || n < 0 || nq < 0 || k < 0 || (nq > 0 && !queries) || !lo_f || !hi_f) return VTO_ERR_ARG;
    vec3 lo = v3(lo_f[0], lo_f[1], lo_f[2]);
    vec3 L = v3((double)hi_f[0] - (double)lo_f[0], (double)hi_f[1] - (double)lo_f[1],
                (double)hi_f[2] - (double)lo_f[2]);
    if (!periodic_ok(L, n)) return VTO_ERR_ARG;
    img_tree* t = img_tree_build(pts, n, lo, L, 0.5 * min3(L));
    const double lim = 0.25 * min3(L) * min3(L) * (1.0 - 1e-9);
    int status = VTO_OK;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        kv* buf = (kv*)malloc((size_t)(k > 0 ? k : 1) * sizeof(kv));
#pragma omp for schedule(dynamic, 256)
        for (int64_t q = 0; q < nq; ++q) {
            int64_t i = queries[q];
            if (i < 0 || i >= n) { status = VTO_ERR_ARG; continue; }
            int m = img_knn(t, i, k, buf);
            kv* use = buf;
            kv* all = NULL;
            if (m < k || (m > 0 && buf[m - 1].d2 >= lim)) {  /* the tree may miss images this far */
                int64_t ma = 0;
                all = img_all(pts, n, L, i, &ma);
                use = all;
                m = ma < k ? (int)ma : k;
            }
            for (int a = 0; a < k; ++a) {
                nbr[q * k + a] = a < m ? (int32_t)(use[a].idx >> 7) : -1;
                if (img) img[q * k + a] = a < m ? (int32_t)(use[a].idx & 127) : -1;
                if (d2) d2[q * k + a] = a < m ? use[a].d2 : INFINITY;
            }
            free(all);
        }
        free(buf);
    }
    img_tree_free(t);
    return status;
}
