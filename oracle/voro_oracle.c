/*
 * FP64 CPU oracle for the cell-based Voronoi method of
 * "An extension to Voro++ for multithreaded computation of Voronoi cells"
 * (arXiv 2209.11606).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 2.1.2):
 *   - the cell of particle P starts as the container box expressed relative
 *     to P, Eqs. (1)-(2): [a-p, b-p] on a walled axis and [-L/2, L/2] on a
 *     periodic axis;
 *   - every other particle (and, on periodic axes, every periodic image) at
 *     relative position q removes the half-space r.q > q.q/2, Eq. (3);
 *     for the radical (power) variant of Sec. 2.1.1 (container_poly) the
 *     removed half-space is r.q > (q.q + r_p^2 - r_q^2)/2 (the standard
 *     power-diagram bisector; the paper names the variant but not the formula);
 *   - applying all of these cuts gives exactly the Voronoi cell (Sec. 2.1.2,
 *     closing paragraph).
 *
 * Two drivers:
 *   method 0 ("brute"): clip by every particle and every image with
 *     |m|_inf <= M.  M starts at 1 and is raised until the stop radius of the
 *     final cell is <= M * L_min, so no omitted image could have cut.
 *   method 1 ("grid"): the Sec. 2.1.3 procedure -- particles are sorted into
 *     the block grid of Sec. 2.1.1, blocks are visited shell by shell outward
 *     from P's own block, and the walk stops at the radius bound: no particle
 *     farther than 2R (R = max vertex distance) can cut the cell.  For the
 *     radical variant the bound is R + sqrt(R^2 + r_max^2 - r_p^2).
 *
 * Cell representation: a list of faces, each a convex polygon of explicit
 * FP64 points in counter-clockwise order seen from outside, tagged with the
 * plane that made it.  A cut is a Sutherland-Hodgman clip of every face plus
 * one new face made of the points that lie on the cutting plane.
 *
 * Conventions where the paper is silent (each is stated in the design notes):
 *   - a vertex with signed distance d = v.q - c <= tau counts as inside
 *     (on-plane vertices stay; Eq. (3) removes only the strict side), with
 *     tau = tau_rel * s * |q|, s = (box volume / N)^(1/dim);
 *   - points closer than merge_rel * s are one vertex (degree > 3 vertices
 *     of exact lattices), faces with fewer than 3 distinct points or of zero
 *     width are dropped and their neighbour is not reported;
 *   - wall faces carry ids -1..-6 (x-, x+, y-, y+, z-, z+); faces of a
 *     periodic box carry the particle's own id with an image shift.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXF 384  /* faces per cell */
#define OR_MAXFV 192 /* vertices per face */
#define OR_MAXNP 1024 /* points on one cutting plane (with duplicates) */
#define OR_MAXV2 1024 /* polygon vertices in 2D */

enum { ST_OK = 0, ST_EMPTY = 1, ST_CAP = 2 };

typedef struct {
    double n[3], c;   /* the cell lies on n.r <= c */
    long long id;     /* neighbour id, or wall code < 0 */
    int img[3];       /* periodic image shift of the neighbour */
    int nv;
    double v[OR_MAXFV][3];
} ofc;

#define OR_MAXX 1024 /* crossing edges of one cut */

typedef struct {
    int nf, cap_hit;
    ofc f[OR_MAXF];
    ofc tmp;
    double np_[OR_MAXNP][3];
    /* per crossing edge of the current cut: its face, its place in the face
     * and the plane of the other face that holds it */
    int nxe, xe_face[OR_MAXX], xe_edge[OR_MAXX];
    double xe_pl[OR_MAXX][4];
} cell3;

typedef struct {
    int nv, cap_hit;
    double v[OR_MAXV2][2];
    long long lid[OR_MAXV2];  /* label of edge v[i] -> v[i+1] */
    int limg[OR_MAXV2][2];
    double ln[OR_MAXV2][3];   /* its line n.x = c: n[0], n[1], c */
    double tv[OR_MAXV2][2];
    long long tlid[OR_MAXV2];
    int timg[OR_MAXV2][2];
    double tln[OR_MAXV2][3];
} cell2;

typedef struct {
    int dim;
    long long n;
    const double *pos, *rad;
    double lo[3], hi[3], L[3];
    int per[3];
    double s, tau_rel, merge_rel, rmax;
    double clip;       /* clipped cells (Sec. 3.1.3): cube side, 0 = none */
    /* grid */
    int nb[3];
    double h[3];
    long long *bstart; /* block CSR, nblk+1 */
    long long *bidx;   /* particle ids sorted by block */
} ctx_t;

/* ---------------------------------------------------------------- helpers */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int lexless(const double *a, const double *b, int d) {
    for (int k = 0; k < d; k++) {
        if (a[k] < b[k]) return 1;
        if (a[k] > b[k]) return 0;
    }
    return 0;
}

/* Point where the segment a-b meets the plane, from the signed distances
 * da, db.  The endpoints are put in lexicographic order first, so that the
 * two faces sharing an edge compute bit-identical points. */
static void isect(const double *a, const double *b, double da, double db, double *x, int d) {
    if (lexless(b, a, d)) {
        const double *t = a; a = b; b = t;
        double tt = da; da = db; db = tt;
    }
    double t = da / (da - db);
    for (int k = 0; k < d; k++) x[k] = a[k] + t * (b[k] - a[k]);
}

static double dist2(const double *a, const double *b, int d) {
    double s = 0;
    for (int k = 0; k < d; k++) s += (a[k] - b[k]) * (a[k] - b[k]);
    return s;
}

/* Sort the points of one plane counter-clockwise about the normal n. */
static void sort_ccw(double (*p)[3], int k, const double *n) {
    double m[3] = {0, 0, 0};
    for (int i = 0; i < k; i++) for (int j = 0; j < 3; j++) m[j] += p[i][j] / k;
    /* u: any unit vector orthogonal to n; w = n x u / |n| */
    double nn = sqrt(dot3(n, n));
    double e[3] = {0, 0, 0};
    int ax = 0;
    if (fabs(n[1]) < fabs(n[ax])) ax = 1;
    if (fabs(n[2]) < fabs(n[ax])) ax = 2;
    e[ax] = 1.0;
    double u[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
    double ul = sqrt(dot3(u, u));
    for (int j = 0; j < 3; j++) u[j] /= ul;
    double w[3] = {(n[1] * u[2] - n[2] * u[1]) / nn, (n[2] * u[0] - n[0] * u[2]) / nn,
                   (n[0] * u[1] - n[1] * u[0]) / nn};
    double ang[OR_MAXNP];
    for (int i = 0; i < k; i++) {
        double r[3] = {p[i][0] - m[0], p[i][1] - m[1], p[i][2] - m[2]};
        ang[i] = atan2(dot3(r, w), dot3(r, u));
    }
    /* insertion sort by angle */
    for (int i = 1; i < k; i++) {
        double a = ang[i], q[3] = {p[i][0], p[i][1], p[i][2]};
        int j = i - 1;
        while (j >= 0 && ang[j] > a) {
            ang[j + 1] = ang[j];
            memcpy(p[j + 1], p[j], sizeof(double) * 3);
            j--;
        }
        ang[j + 1] = a;
        memcpy(p[j + 1], q, sizeof(double) * 3);
    }
}

/* Remove consecutive (cyclic) points closer than eps; returns the new count. */
static int dedupe_cyclic3(double (*p)[3], int k, double eps2) {
    int m = 0;
    for (int i = 0; i < k; i++) {
        if (m > 0 && dist2(p[i], p[m - 1], 3) <= eps2) continue;
        if (m != i) memcpy(p[m], p[i], sizeof(double) * 3);
        m++;
    }
    while (m > 1 && dist2(p[m - 1], p[0], 3) <= eps2) m--;
    return m;
}

/* A face is kept only with >= 3 points and a width above eps:
 * |vector area| > eps * perimeter. */
static int face_ok(double (*p)[3], int k, double eps) {
    if (k < 3) return 0;
    double A[3] = {0, 0, 0}, per = 0;
    for (int i = 1; i + 1 < k; i++) {
        double a[3], b[3];
        for (int j = 0; j < 3; j++) { a[j] = p[i][j] - p[0][j]; b[j] = p[i + 1][j] - p[0][j]; }
        A[0] += a[1] * b[2] - a[2] * b[1];
        A[1] += a[2] * b[0] - a[0] * b[2];
        A[2] += a[0] * b[1] - a[1] * b[0];
    }
    for (int i = 0; i < k; i++) per += sqrt(dist2(p[i], p[(i + 1) % k], 3));
    return 0.5 * sqrt(dot3(A, A)) > eps * per;
}

/* ------------------------------------------------------------ 3D cell */

/* Initial cell, Eqs. (1)-(2): the box relative to particle p. */
/* Initial cell bounds relative to p along each axis (Eqs. (1)-(2)): the box,
 * or half the period on a periodic axis.  A clipped cell (Sec. 3.1.3) starts
 * from the intersection with the cube of side `clip` centred on p; a face
 * the cube supplies is a wall face (wall[a] set for a periodic axis whose
 * half period exceeds the half side). */
static void init_bounds(const ctx_t *cx, const double *p, int d, double *lo, double *hi, int *wall) {
    for (int a = 0; a < d; a++) {
        wall[a] = !cx->per[a];
        if (cx->per[a]) { lo[a] = -0.5 * cx->L[a]; hi[a] = 0.5 * cx->L[a]; }
        else { lo[a] = cx->lo[a] - p[a]; hi[a] = cx->hi[a] - p[a]; }
        if (cx->clip > 0) {
            const double hc = 0.5 * cx->clip;
            if (cx->per[a]) {
                if (hc < hi[a]) { lo[a] = -hc; hi[a] = hc; wall[a] = 1; }
            } else {
                if (-hc > lo[a]) lo[a] = -hc;
                if (hc < hi[a]) hi[a] = hc;
            }
        }
    }
}

static void init3(cell3 *cl, const ctx_t *cx, const double *p, long long self) {
    double lo[3], hi[3];
    int wall[3];
    init_bounds(cx, p, 3, lo, hi, wall);
    cl->nf = 0;
    cl->cap_hit = 0;
    for (int a = 0; a < 3; a++) {
        for (int side = 0; side < 2; side++) {
            ofc *f = &cl->f[cl->nf++];
            memset(f->n, 0, sizeof f->n);
            f->n[a] = side ? 1.0 : -1.0;
            f->c = side ? hi[a] : -lo[a];
            f->img[0] = f->img[1] = f->img[2] = 0;
            if (!wall[a]) { f->id = self; f->img[a] = side ? 1 : -1; }
            else f->id = -(1 + 2 * a + side);
            int b = (a + 1) % 3, c = (a + 2) % 3, k = 0;
            for (int ib = 0; ib < 2; ib++)
                for (int ic = 0; ic < 2; ic++) {
                    f->v[k][a] = side ? hi[a] : lo[a];
                    f->v[k][b] = ib ? hi[b] : lo[b];
                    f->v[k][c] = ic ? hi[c] : lo[c];
                    k++;
                }
            f->nv = 4;
            sort_ccw(f->v, 4, f->n);
        }
    }
}

static int same3(const double *a, const double *b) { return a[0] == b[0] && a[1] == b[1] && a[2] == b[2]; }

/* Where the edge a-b, on the planes p1 and p2 (n, c each), crosses the cut
 * plane q.r = c: the point on all three planes (Cramer's rule), so that its
 * error is relative to the cell, not to the edge, which at first is as long
 * as the box.  The two edge planes are taken in lexicographic order, so the
 * two faces that share the edge compute the same point; nearly dependent
 * planes fall back to interpolating along the edge. */
static void cross3p(const double *p1, const double *p2, const double *q, double c, const double *a, const double *b,
                    double da, double db, double *x) {
    const double *u = p1, *w = p2;
    for (int k = 0; k < 4; k++) {
        if (p1[k] < p2[k]) break;
        if (p1[k] > p2[k]) { u = p2; w = p1; break; }
    }
    const double wq[3] = {w[1] * q[2] - w[2] * q[1], w[2] * q[0] - w[0] * q[2], w[0] * q[1] - w[1] * q[0]};
    const double qu[3] = {q[1] * u[2] - q[2] * u[1], q[2] * u[0] - q[0] * u[2], q[0] * u[1] - q[1] * u[0]};
    const double uw[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    const double det = u[0] * wq[0] + u[1] * wq[1] + u[2] * wq[2];
    if (fabs(det) <= 1e-6 * sqrt(dot3(u, u) * dot3(w, w) * dot3(q, q))) {
        isect(a, b, da, db, x, 3);
        return;
    }
    for (int k = 0; k < 3; k++) x[k] = (u[3] * wq[k] + w[3] * qu[k] + c * uw[k]) / det;
}

/* Cut the cell by { r : q.r > c } (Eq. (3)).  Returns 0 if nothing was
 * removed, 1 if the cell changed, 2 if it became empty. */
static int clip3(cell3 *cl, const double *q, double c, double tau, double eps,
                 long long id, const int *img) {
    int any = 0;
    for (int i = 0; i < cl->nf && !any; i++)
        for (int j = 0; j < cl->f[i].nv; j++)
            if (dot3(q, cl->f[i].v[j]) - c > tau) { any = 1; break; }
    if (!any) return 0;
    /* the crossing edges and, before any face changes, the plane of the
     * other face holding each (traversed the other way) */
    cl->nxe = 0;
    for (int i = 0; i < cl->nf; i++) {
        const ofc *f = &cl->f[i];
        for (int j = 0; j < f->nv; j++) {
            const double *a = f->v[j], *b = f->v[(j + 1) % f->nv];
            const double da = dot3(q, a) - c, db = dot3(q, b) - c;
            if (!((da > tau && db < -tau) || (da < -tau && db > tau)) || cl->nxe >= OR_MAXX) continue;
            int g = -1;
            for (int i2 = 0; i2 < cl->nf && g < 0; i2++) {
                if (i2 == i) continue;
                const ofc *h = &cl->f[i2];
                for (int j2 = 0; j2 < h->nv; j2++)
                    if (same3(h->v[j2], b) && same3(h->v[(j2 + 1) % h->nv], a)) { g = i2; break; }
            }
            if (g < 0) continue;
            const int t = cl->nxe++;
            cl->xe_face[t] = i;
            cl->xe_edge[t] = j;
            cl->xe_pl[t][0] = cl->f[g].n[0]; cl->xe_pl[t][1] = cl->f[g].n[1];
            cl->xe_pl[t][2] = cl->f[g].n[2]; cl->xe_pl[t][3] = cl->f[g].c;
        }
    }
    double eps2 = eps * eps;
    int npn = 0, nf = 0;
    for (int i = 0; i < cl->nf; i++) {
        ofc *f = &cl->f[i];
        ofc *o = &cl->tmp;
        int k = 0;
        for (int j = 0; j < f->nv; j++) {
            const double *a = f->v[j], *b = f->v[(j + 1) % f->nv];
            double da = dot3(q, a) - c, db = dot3(q, b) - c;
            if (da <= tau) {
                if (k < OR_MAXFV) memcpy(o->v[k], a, sizeof(double) * 3);
                k++;
                if (fabs(da) <= tau) {
                    if (npn < OR_MAXNP) memcpy(cl->np_[npn], a, sizeof(double) * 3);
                    npn++;
                }
            }
            if ((da > tau && db < -tau) || (da < -tau && db > tau)) {
                double x[3];
                int t = 0;
                while (t < cl->nxe && !(cl->xe_face[t] == i && cl->xe_edge[t] == j)) t++;
                if (t < cl->nxe) {
                    const double pf[4] = {f->n[0], f->n[1], f->n[2], f->c};
                    cross3p(pf, cl->xe_pl[t], q, c, a, b, da, db, x);
                } else {
                    isect(a, b, da, db, x, 3);
                }
                if (k < OR_MAXFV) memcpy(o->v[k], x, sizeof(double) * 3);
                k++;
                if (npn < OR_MAXNP) memcpy(cl->np_[npn], x, sizeof(double) * 3);
                npn++;
            }
        }
        if (k > OR_MAXFV || npn > OR_MAXNP) { cl->cap_hit = 1; return 1; }
        k = dedupe_cyclic3(o->v, k, eps2);
        if (!face_ok(o->v, k, eps)) continue;
        ofc *d = &cl->f[nf++];
        if (d != f) { memcpy(d->n, f->n, sizeof f->n); d->c = f->c; d->id = f->id; memcpy(d->img, f->img, sizeof f->img); }
        d->nv = k;
        memcpy(d->v, o->v, sizeof(double) * 3 * k);
    }
    cl->nf = nf;
    /* the new face: the distinct points on the cutting plane */
    int m = 0;
    for (int i = 0; i < npn; i++) {
        int dup = 0;
        for (int j = 0; j < m && !dup; j++) dup = dist2(cl->np_[i], cl->np_[j], 3) <= eps2;
        if (!dup) { if (m != i) memcpy(cl->np_[m], cl->np_[i], sizeof(double) * 3); m++; }
    }
    if (m >= 3) {
        sort_ccw(cl->np_, m, q);
        m = dedupe_cyclic3(cl->np_, m, eps2);
        if (face_ok(cl->np_, m, eps)) {
            if (cl->nf >= OR_MAXF || m > OR_MAXFV) { cl->cap_hit = 1; return 1; }
            ofc *d = &cl->f[cl->nf++];
            memcpy(d->n, q, sizeof(double) * 3);
            d->c = c;
            d->id = id;
            d->img[0] = img[0]; d->img[1] = img[1]; d->img[2] = img[2];
            d->nv = m;
            memcpy(d->v, cl->np_, sizeof(double) * 3 * m);
        }
    }
    return cl->nf == 0 ? 2 : 1;
}

static double maxr3(const cell3 *cl) {
    double r2 = 0;
    for (int i = 0; i < cl->nf; i++)
        for (int j = 0; j < cl->f[i].nv; j++) {
            double t = dot3(cl->f[i].v[j], cl->f[i].v[j]);
            if (t > r2) r2 = t;
        }
    return sqrt(r2);
}

/* ------------------------------------------------------------ 2D cell */

static void init2(cell2 *cl, const ctx_t *cx, const double *p, long long self) {
    double lo[2], hi[2];
    int wall[2];
    init_bounds(cx, p, 2, lo, hi, wall);
    /* counter-clockwise: bottom (y-), right (x+), top (y+), left (x-) */
    double vx[4] = {lo[0], hi[0], hi[0], lo[0]}, vy[4] = {lo[1], lo[1], hi[1], hi[1]};
    int ax[4] = {1, 0, 1, 0}, sd[4] = {0, 1, 1, 0};
    cl->nv = 4;
    cl->cap_hit = 0;
    for (int i = 0; i < 4; i++) {
        cl->v[i][0] = vx[i];
        cl->v[i][1] = vy[i];
        int a = ax[i], s = sd[i];
        cl->limg[i][0] = cl->limg[i][1] = 0;
        if (!wall[a]) { cl->lid[i] = self; cl->limg[i][a] = s ? 1 : -1; }
        else cl->lid[i] = -(1 + 2 * a + s);
        cl->ln[i][0] = a == 0 ? (s ? 1.0 : -1.0) : 0.0;
        cl->ln[i][1] = a == 1 ? (s ? 1.0 : -1.0) : 0.0;
        cl->ln[i][2] = s ? hi[a] : -lo[a];
    }
}

/* Where the edge a-b, on the line n.x = n[2], crosses the cut line
 * q.x = c: the point on both lines (Cramer's rule), so that its error is
 * relative to the cell, not to the edge, which at first is as long as the
 * box; nearly parallel lines fall back to interpolating along the edge. */
static void cross2(const double *n, const double *q, double c, const double *a, const double *b, double da,
                   double db, double *x) {
    const double det = n[0] * q[1] - n[1] * q[0];
    const double nn = sqrt(n[0] * n[0] + n[1] * n[1]), qn = sqrt(q[0] * q[0] + q[1] * q[1]);
    if (fabs(det) <= 1e-6 * nn * qn) {
        isect(a, b, da, db, x, 2);
        return;
    }
    x[0] = (n[2] * q[1] - c * n[1]) / det;
    x[1] = (n[0] * c - q[0] * n[2]) / det;
}

static void setln(double *dst, const double *src) { dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; }

static int clip2(cell2 *cl, const double *q, double c, double tau, double eps,
                 long long id, const int *img) {
    const double qc[3] = {q[0], q[1], c};
    int any = 0;
    for (int j = 0; j < cl->nv; j++)
        if (q[0] * cl->v[j][0] + q[1] * cl->v[j][1] - c > tau) { any = 1; break; }
    if (!any) return 0;
    int k = 0, n = cl->nv;
    for (int j = 0; j < n; j++) {
        const double *a = cl->v[j], *b = cl->v[(j + 1) % n];
        double da = q[0] * a[0] + q[1] * a[1] - c, db = q[0] * b[0] + q[1] * b[1] - c;
        if (k + 2 > OR_MAXV2) { cl->cap_hit = 1; return 1; }
        if (da <= tau) {
            /* a stays; the edge leaving it follows the cut line if b is out */
            cl->tv[k][0] = a[0]; cl->tv[k][1] = a[1];
            if (db > tau) { cl->tlid[k] = id; cl->timg[k][0] = img[0]; cl->timg[k][1] = img[1]; setln(cl->tln[k], qc); }
            else {
                cl->tlid[k] = cl->lid[j]; cl->timg[k][0] = cl->limg[j][0]; cl->timg[k][1] = cl->limg[j][1];
                setln(cl->tln[k], cl->ln[j]);
            }
            k++;
            if (da < -tau && db > tau) {
                /* leaving: the crossing point, then along the cut line */
                cross2(cl->ln[j], q, c, a, b, da, db, cl->tv[k]);
                cl->tlid[k] = id; cl->timg[k][0] = img[0]; cl->timg[k][1] = img[1]; setln(cl->tln[k], qc);
                /* the edge a->x keeps the old label, x->... follows the cut */
                cl->tlid[k - 1] = cl->lid[j]; cl->timg[k - 1][0] = cl->limg[j][0]; cl->timg[k - 1][1] = cl->limg[j][1];
                setln(cl->tln[k - 1], cl->ln[j]);
                k++;
            }
        } else if (db < -tau) {
            /* entering: the crossing point, then along the old edge */
            cross2(cl->ln[j], q, c, a, b, da, db, cl->tv[k]);
            cl->tlid[k] = cl->lid[j]; cl->timg[k][0] = cl->limg[j][0]; cl->timg[k][1] = cl->limg[j][1];
            setln(cl->tln[k], cl->ln[j]);
            k++;
        }
    }
    /* merge coincident neighbours: keep the first point, the second's label */
    double eps2 = eps * eps;
    int m = 0;
    for (int i = 0; i < k; i++) {
        if (m > 0 && dist2(cl->tv[i], cl->v[m - 1], 2) <= eps2) {
            cl->lid[m - 1] = cl->tlid[i]; cl->limg[m - 1][0] = cl->timg[i][0]; cl->limg[m - 1][1] = cl->timg[i][1];
            setln(cl->ln[m - 1], cl->tln[i]);
            continue;
        }
        cl->v[m][0] = cl->tv[i][0]; cl->v[m][1] = cl->tv[i][1];
        cl->lid[m] = cl->tlid[i]; cl->limg[m][0] = cl->timg[i][0]; cl->limg[m][1] = cl->timg[i][1];
        setln(cl->ln[m], cl->tln[i]);
        m++;
    }
    while (m > 1 && dist2(cl->v[m - 1], cl->v[0], 2) <= eps2) {
        /* the last point coincides with the first: drop it and its zero edge */
        m--;
    }
    /* a polygon thinner than eps is empty */
    if (m < 3) { cl->nv = 0; return 2; }
    double A = 0, per = 0;
    for (int i = 0; i < m; i++) {
        int j = (i + 1) % m;
        A += cl->v[i][0] * cl->v[j][1] - cl->v[j][0] * cl->v[i][1];
        per += sqrt(dist2(cl->v[i], cl->v[j], 2));
    }
    if (0.5 * fabs(A) <= eps * per) { cl->nv = 0; return 2; }
    cl->nv = m;
    return 1;
}

static double maxr2(const cell2 *cl) {
    double r2 = 0;
    for (int j = 0; j < cl->nv; j++) {
        double t = cl->v[j][0] * cl->v[j][0] + cl->v[j][1] * cl->v[j][1];
        if (t > r2) r2 = t;
    }
    return sqrt(r2);
}

/* --------------------------------------------------------- one candidate */

typedef struct {
    cell3 *c3;
    cell2 *c2;
    double p[3], rp;
    long long self;
    long long ntested, ncut;
} job_t;

/* Radius bound (Sec. 2.1.3): no particle farther than this can cut. */
static double stop_radius(const ctx_t *cx, const job_t *jb) {
    double R = cx->dim == 3 ? maxr3(jb->c3) : maxr2(jb->c2);
    if (!cx->rad) return 2.0 * R;
    double disc = R * R + cx->rmax * cx->rmax - jb->rp * jb->rp;
    return disc > 0 ? R + sqrt(disc) : 0.0;
}

/* Apply the cut of particle j with image shift m.  Returns the clip code. */
static int apply(const ctx_t *cx, job_t *jb, long long j, const int *m) {
    int d = cx->dim;
    double q[3] = {0, 0, 0}, qq = 0;
    for (int a = 0; a < d; a++) {
        q[a] = (cx->pos[j * d + a] + m[a] * cx->L[a]) - jb->p[a];
        qq += q[a] * q[a];
    }
    double rj = cx->rad ? cx->rad[j] : 0.0;
    double c = 0.5 * (qq + jb->rp * jb->rp - rj * rj);
    double tau = cx->tau_rel * cx->s * sqrt(qq);
    double eps = cx->merge_rel * cx->s;
    jb->ntested++;
    int r = d == 3 ? clip3(jb->c3, q, c, tau, eps, j, m) : clip2(jb->c2, q, c, tau, eps, j, m);
    if (r) jb->ncut++;
    return r;
}

/* ------------------------------------------------------------- drivers */

/* Brute force: every particle, every image with |m|_inf <= M. */
static int cell_brute(const ctx_t *cx, job_t *jb) {
    int d = cx->dim;
    double Lmin = INFINITY;
    int anyper = 0;
    for (int a = 0; a < d; a++) if (cx->per[a]) { anyper = 1; if (cx->L[a] < Lmin) Lmin = cx->L[a]; }
    for (int M = 1;; M++) {
        if (d == 3) init3(jb->c3, cx, jb->p, jb->self); else init2(jb->c2, cx, jb->p, jb->self);
        jb->ntested = jb->ncut = 0;
        int ext[3];
        for (int a = 0; a < 3; a++) ext[a] = (a < d && cx->per[a]) ? M : 0;
        int empty = 0;
        for (long long j = 0; j < cx->n && !empty; j++)
            for (int mx = -ext[0]; mx <= ext[0] && !empty; mx++)
                for (int my = -ext[1]; my <= ext[1] && !empty; my++)
                    for (int mz = -ext[2]; mz <= ext[2] && !empty; mz++) {
                        if (j == jb->self && mx == 0 && my == 0 && mz == 0) continue;
                        int m[3] = {mx, my, mz};
                        if (apply(cx, jb, j, m) == 2) empty = 1;
                    }
        if (empty) return ST_EMPTY;
        if ((d == 3 ? jb->c3->cap_hit : jb->c2->cap_hit)) return ST_CAP;
        if (!anyper || stop_radius(cx, jb) <= M * Lmin) return ST_OK;
    }
}

static int floordiv(int a, int b) { int q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }

/* Grid walk (Sec. 2.1.3): own block first, then Chebyshev shells outward;
 * a block is skipped if its nearest point is beyond the stop radius, and the
 * walk ends once a whole shell lies beyond it. */
static int cell_grid(const ctx_t *cx, job_t *jb, const int *bp) {
    int d = cx->dim;
    if (d == 3) init3(jb->c3, cx, jb->p, jb->self); else init2(jb->c2, cx, jb->p, jb->self);
    jb->ntested = jb->ncut = 0;
    double hmin = INFINITY;
    int maxn = 0;
    for (int a = 0; a < d; a++) { if (cx->h[a] < hmin) hmin = cx->h[a]; if (cx->nb[a] > maxn) maxn = cx->nb[a]; }
    double rs = stop_radius(cx, jb);
    for (int s = 0;; s++) {
        if (s >= 1 && (s - 1) * hmin >= rs) break;
        int anyper = 0;
        for (int a = 0; a < d; a++) anyper |= cx->per[a];
        if (!anyper && s > maxn) break;
        int lim[3] = {0, 0, 0};
        for (int a = 0; a < d; a++) lim[a] = s;
        for (int ox = -lim[0]; ox <= lim[0]; ox++)
            for (int oy = -lim[1]; oy <= lim[1]; oy++)
                for (int oz = -lim[2]; oz <= lim[2]; oz++) {
                    int o[3] = {ox, oy, oz};
                    int cheb = 0;
                    for (int a = 0; a < d; a++) if (abs(o[a]) > cheb) cheb = abs(o[a]);
                    if (cheb != s) continue;
                    int t[3] = {0, 0, 0}, m[3] = {0, 0, 0}, ok = 1;
                    double dd = 0;
                    for (int a = 0; a < d && ok; a++) {
                        int ta = bp[a] + o[a];
                        if (cx->per[a]) { m[a] = floordiv(ta, cx->nb[a]); ta -= m[a] * cx->nb[a]; }
                        else if (ta < 0 || ta >= cx->nb[a]) { ok = 0; break; }
                        t[a] = ta;
                        /* the block's extent relative to p */
                        double blo = cx->lo[a] + ta * cx->h[a] + m[a] * cx->L[a] - jb->p[a];
                        double bhi = blo + cx->h[a];
                        double g = blo > 0 ? blo : (bhi < 0 ? -bhi : 0.0);
                        dd += g * g;
                    }
                    if (!ok) continue;
                    if (sqrt(dd) >= rs) continue;
                    long long k = t[0] + (long long)cx->nb[0] * (t[1] + (long long)cx->nb[1] * t[2]);
                    for (long long u = cx->bstart[k]; u < cx->bstart[k + 1]; u++) {
                        long long j = cx->bidx[u];
                        if (j == jb->self && m[0] == 0 && m[1] == 0 && m[2] == 0) continue;
                        int r = apply(cx, jb, j, m);
                        if (r == 2) return ST_EMPTY;
                        if (r == 1) rs = stop_radius(cx, jb);
                    }
                }
    }
    if ((d == 3 ? jb->c3->cap_hit : jb->c2->cap_hit)) return ST_CAP;
    return ST_OK;
}

/* ------------------------------------------------------------ statistics */

typedef struct {
    double vol, area, cen[3], R;
    int nv, ne, nf;
    /* Weinberg code of the edge graph (Sec. 4): darts traversed (2E, 0 when
     * not computed), FNV-1a 64 hash of the 2E+1 vertex labels (each label
     * as two little-endian bytes), number of (start, orientation) pairs that
     * give the minimal code */
    int wlen, wsym;
    unsigned long long whash;
} stats_t;

/* Weinberg's traversal of a planar graph given by its darts (from, to), the
 * reverse of each dart and a rotation rot[d]: the next dart leaving from[d]
 * in cyclic order.  From a start dart, arriving at y by dart d: at a new
 * vertex leave by the next dart after the reverse of d; at an old vertex
 * return along the reverse of d if it is untraversed, else leave by the
 * first untraversed dart after the reverse of d.  The code lists the labels
 * (order of first visit, from 1) of the start and of every arrival, 2E + 1
 * entries.  The cell's code is the lexicographic minimum over every start
 * dart and both rotation directions; `sym` counts the pairs that reach it.
 * Returns 0 if some traversal ends before using every dart. */
static int weinberg(int V, int D, const int *dfrom, const int *dto, const int *rev, const int *rot,
                    const int *rotinv, int *best, int *cur, int *lab, unsigned char *used, int *sym) {
    int have = 0;
    *sym = 0;
    for (int o = 0; o < 2; o++) {
        const int *R = o ? rotinv : rot;
        for (int s0 = 0; s0 < D; s0++) {
            for (int v = 0; v < V; v++) lab[v] = 0;
            memset(used, 0, (size_t)D);
            int nl = 1, d = s0;
            lab[dfrom[s0]] = nl;
            cur[0] = 1;
            for (int k = 0; k < D; k++) {
                used[d] = 1;
                const int y = dto[d];
                int nd = -1;
                if (!lab[y]) {
                    lab[y] = ++nl;
                    nd = R[rev[d]];
                } else if (!used[rev[d]]) {
                    nd = rev[d];
                } else {
                    int e = R[rev[d]];
                    while (used[e] && e != rev[d]) e = R[e];
                    if (!used[e]) nd = e;
                }
                cur[k + 1] = lab[y];
                if (k + 1 < D) {
                    if (nd < 0) return 0;
                    d = nd;
                }
            }
            int c = 0;
            if (have)
                for (int k = 0; k <= D && !c; k++) c = cur[k] < best[k] ? -1 : (cur[k] > best[k] ? 1 : 0);
            if (!have || c < 0) {
                memcpy(best, cur, sizeof(int) * (size_t)(D + 1));
                have = 1;
                *sym = 1;
            } else if (c == 0) {
                (*sym)++;
            }
        }
    }
    return 1;
}

static unsigned long long fnv1a_labels(const int *code, int n) {
    unsigned long long h = 14695981039346656037ull;
    for (int k = 0; k < n; k++) {
        h ^= (unsigned long long)(code[k] & 0xff);
        h *= 1099511628211ull;
        h ^= (unsigned long long)((code[k] >> 8) & 0xff);
        h *= 1099511628211ull;
    }
    return h;
}

/* 3D: volume and centroid by fans from each face's first vertex to a fixed
 * apex o (the tetrahedral decomposition of a closed surface does not depend
 * on the apex; a vertex of the cell is used so that a radical cell lying far
 * from its particle does not cancel); area = sum of face areas; V, E by
 * merging coincident points (eps) over all faces. */
static void stats3(const cell3 *cl, double eps, stats_t *st, int *forder) {
    double vol = 0, cx = 0, cy = 0, cz = 0, area = 0;
    const double *o = cl->nf > 0 ? cl->f[0].v[0] : NULL;
    for (int i = 0; i < cl->nf; i++) {
        const ofc *f = &cl->f[i];
        double A[3] = {0, 0, 0};
        for (int j = 1; j + 1 < f->nv; j++) {
            const double a[3] = {f->v[0][0] - o[0], f->v[0][1] - o[1], f->v[0][2] - o[2]};
            const double b[3] = {f->v[j][0] - o[0], f->v[j][1] - o[1], f->v[j][2] - o[2]};
            const double c[3] = {f->v[j + 1][0] - o[0], f->v[j + 1][1] - o[1], f->v[j + 1][2] - o[2]};
            double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                         a[2] * (b[0] * c[1] - b[1] * c[0]);
            double v6 = det / 6.0;
            vol += v6;
            cx += v6 * (a[0] + b[0] + c[0]) / 4.0;
            cy += v6 * (a[1] + b[1] + c[1]) / 4.0;
            cz += v6 * (a[2] + b[2] + c[2]) / 4.0;
            double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            A[0] += e1[1] * e2[2] - e1[2] * e2[1];
            A[1] += e1[2] * e2[0] - e1[0] * e2[2];
            A[2] += e1[0] * e2[1] - e1[1] * e2[0];
        }
        area += 0.5 * sqrt(dot3(A, A));
        forder[i] = f->nv;
    }
    st->vol = vol;
    st->area = area;
    st->cen[0] = vol != 0 ? o[0] + cx / vol : 0;
    st->cen[1] = vol != 0 ? o[1] + cy / vol : 0;
    st->cen[2] = vol != 0 ? o[2] + cz / vol : 0;
    st->nf = cl->nf;
    /* distinct vertices */
    int tot = 0;
    for (int i = 0; i < cl->nf; i++) tot += cl->f[i].nv;
    const double **pts = (const double **)malloc(sizeof(double *) * (tot ? tot : 1));
    int *cid = (int *)malloc(sizeof(int) * (tot ? tot : 1));
    int k = 0, nv = 0;
    double eps2 = eps * eps;
    for (int i = 0; i < cl->nf; i++)
        for (int j = 0; j < cl->f[i].nv; j++) {
            pts[k] = cl->f[i].v[j];
            cid[k] = -1;
            for (int u = 0; u < k; u++)
                if (dist2(pts[u], pts[k], 3) <= eps2) { cid[k] = cid[u]; break; }
            if (cid[k] < 0) cid[k] = nv++;
            k++;
        }
    /* distinct edges: pairs of consecutive cluster ids */
    int ne = 0;
    int *ea = (int *)malloc(sizeof(int) * (tot ? tot : 1)), *eb = (int *)malloc(sizeof(int) * (tot ? tot : 1));
    k = 0;
    for (int i = 0; i < cl->nf; i++) {
        int nvf = cl->f[i].nv;
        for (int j = 0; j < nvf; j++) {
            int a = cid[k + j], b = cid[k + (j + 1) % nvf];
            if (a == b) continue;
            int lo = a < b ? a : b, hi = a < b ? b : a, seen = 0;
            for (int u = 0; u < ne && !seen; u++) seen = (ea[u] == lo && eb[u] == hi);
            if (!seen) { ea[ne] = lo; eb[ne] = hi; ne++; }
        }
        k += nvf;
    }
    st->nv = nv;
    st->ne = ne;
    st->R = maxr3(cl);
    /* darts of the merged face cycles (faces are counterclockwise seen from
     * outside, so each dart lies on exactly one face); rot(v->w) = (v->u) with
     * u the vertex before v on the face of v->w */
    st->wlen = 0; st->wsym = 0; st->whash = 0;
    {
        int D = 0;
        int *df = (int *)malloc(sizeof(int) * (tot ? tot : 1)), *dt = (int *)malloc(sizeof(int) * (tot ? tot : 1));
        int *dp = (int *)malloc(sizeof(int) * (tot ? tot : 1));
        k = 0;
        int ok = 1;
        for (int i = 0; i < cl->nf; i++) {
            const int nvf = cl->f[i].nv;
            int cyc[OR_MAXFV], m = 0;
            for (int j = 0; j < nvf; j++) {
                const int c = cid[k + j];
                if (m == 0 || cyc[m - 1] != c) cyc[m++] = c;
            }
            while (m > 1 && cyc[m - 1] == cyc[0]) m--;
            k += nvf;
            if (m < 3) continue;  /* a face merged away */
            for (int j = 0; j < m; j++) {
                df[D] = cyc[j]; dt[D] = cyc[(j + 1) % m]; dp[D] = cyc[(j + m - 1) % m];
                D++;
            }
        }
        int *rev = (int *)malloc(sizeof(int) * (D ? D : 1)), *rot = (int *)malloc(sizeof(int) * (D ? D : 1));
        int *rinv = (int *)malloc(sizeof(int) * (D ? D : 1));
        for (int d = 0; d < D && ok; d++) {
            rev[d] = rot[d] = -1;
            for (int e = 0; e < D; e++) {
                if (df[e] == dt[d] && dt[e] == df[d]) rev[d] = e;
                if (df[e] == df[d] && dt[e] == dp[d]) rot[d] = e;
            }
            if (rev[d] < 0 || rot[d] < 0) ok = 0;
        }
        if (ok && D == 2 * ne) {
            for (int d = 0; d < D; d++) rinv[rot[d]] = d;
            int *best = (int *)malloc(sizeof(int) * (D + 1)), *curc = (int *)malloc(sizeof(int) * (D + 1));
            int *labv = (int *)malloc(sizeof(int) * (nv ? nv : 1));
            unsigned char *used = (unsigned char *)malloc((size_t)(D ? D : 1));
            int sym = 0;
            if (weinberg(nv, D, df, dt, rev, rot, rinv, best, curc, labv, used, &sym)) {
                st->wlen = D;
                st->wsym = sym;
                st->whash = fnv1a_labels(best, D + 1);
            }
            free(best); free(curc); free(labv); free(used);
        }
        free(df); free(dt); free(dp); free(rev); free(rot); free(rinv);
    }
    free(pts); free(cid); free(ea); free(eb);
}

/* 2D: shoelace sums taken about the first vertex o (translation does not
 * change them; it avoids cancellation for cells far from their particle). */
static void stats2(const cell2 *cl, stats_t *st) {
    double A = 0, cx = 0, cy = 0, per = 0;
    int n = cl->nv;
    const double o[2] = {n ? cl->v[0][0] : 0.0, n ? cl->v[0][1] : 0.0};
    for (int i = 0; i < n; i++) {
        int j = (i + 1) % n;
        const double ax = cl->v[i][0] - o[0], ay = cl->v[i][1] - o[1];
        const double bx = cl->v[j][0] - o[0], by = cl->v[j][1] - o[1];
        double cr = ax * by - bx * ay;
        A += cr / 2.0;
        cx += cr * (ax + bx) / 6.0;
        cy += cr * (ay + by) / 6.0;
        per += sqrt(dist2(cl->v[i], cl->v[j], 2));
    }
    st->vol = A;
    st->area = per;
    st->cen[0] = A != 0 ? o[0] + cx / A : 0;
    st->cen[1] = A != 0 ? o[1] + cy / A : 0;
    st->cen[2] = 0;
    st->nv = st->ne = st->nf = n;
    st->R = maxr2(cl);
}

/* ------------------------------------------------------------ public API */

/*
 * Compute the cells `cells[0..ncell)` (NULL: all n) of the n particles at
 * `pos` (n x dim, FP64) in the box [lo, hi] with the given periodic flags.
 * `radii` (NULL: plain Voronoi) selects the radical variant.  `method` 0 is
 * the brute-force definition, 1 the block-grid walk with `nblocks` blocks.
 * `wlen`, `whash`, `wsym` (NULL: skipped) receive each 3D cell's Weinberg
 * code (Sec. 4): darts traversed, hash of the minimal code and its count.
 * `clip` > 0 gives clipped cells (Sec. 3.1.3): each cell starts from the
 * box intersected with the cube of side `clip` centred on its particle, and
 * the cube's faces are reported as walls.  Per-cell outputs are indexed by position in `cells`; faces go to slabs of
 * `maxf` entries per cell (id, image shift x3, face order), in canonical
 * order: ascending (id, image shift).  Returns 0, or -1 on bad arguments.
 */
int vo_compute(int dim, long long n, const double *pos, const double *radii,
               const double *lo, const double *hi, const int *periodic,
               int method, const int *nblocks, double tau_rel, double merge_rel, double clip,
               long long ncell, const long long *cells, int maxf,
               double *vol, double *area, double *cen, int *nv, int *ne, int *nf,
               int *status, long long *nbr_id, int *nbr_img, int *face_order,
               double *rmax, long long *ntested, long long *ncut, int nthreads,
               int *wlen, unsigned long long *whash, int *wsym) {
    if ((dim != 2 && dim != 3) || n < 0 || !pos || maxf <= 0) return -1;
    ctx_t cx;
    memset(&cx, 0, sizeof cx);
    cx.dim = dim;
    cx.n = n;
    cx.pos = pos;
    cx.rad = radii;
    double V = 1;
    for (int a = 0; a < dim; a++) {
        cx.lo[a] = lo[a]; cx.hi[a] = hi[a]; cx.L[a] = hi[a] - lo[a]; cx.per[a] = periodic[a] != 0;
        V *= cx.L[a];
    }
    cx.s = pow(V / (n > 0 ? (double)n : 1.0), 1.0 / dim);
    cx.tau_rel = tau_rel;
    cx.merge_rel = merge_rel;
    cx.clip = clip > 0 ? clip : 0.0;
    cx.rmax = 0;
    if (radii) for (long long i = 0; i < n; i++) if (radii[i] > cx.rmax) cx.rmax = radii[i];
    long long nblk = 1;
    if (method == 1) {
        for (int a = 0; a < dim; a++) {
            if (nblocks[a] < 1) return -1;
            cx.nb[a] = nblocks[a];
            cx.h[a] = cx.L[a] / nblocks[a];
            nblk *= nblocks[a];
        }
        /* counting sort of particle ids into blocks (Sec. 2.1.1) */
        cx.bstart = (long long *)calloc((size_t)nblk + 1, sizeof(long long));
        cx.bidx = (long long *)malloc(sizeof(long long) * (size_t)(n ? n : 1));
        long long *bk = (long long *)malloc(sizeof(long long) * (size_t)(n ? n : 1));
        for (long long i = 0; i < n; i++) {
            long long k = 0, mul = 1;
            for (int a = 0; a < dim; a++) {
                int b = (int)floor((pos[i * dim + a] - lo[a]) / cx.h[a]);
                if (b < 0) b = 0;
                if (b >= cx.nb[a]) b = cx.nb[a] - 1;
                k += mul * b;
                mul *= cx.nb[a];
            }
            bk[i] = k;
            cx.bstart[k + 1]++;
        }
        for (long long k = 0; k < nblk; k++) cx.bstart[k + 1] += cx.bstart[k];
        long long *fill = (long long *)calloc((size_t)nblk, sizeof(long long));
        for (long long i = 0; i < n; i++) cx.bidx[cx.bstart[bk[i]] + fill[bk[i]]++] = i;
        free(fill);
        free(bk);
    }
    if (ncell < 0) ncell = n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
    {
        job_t jb;
        memset(&jb, 0, sizeof jb);
        if (dim == 3) jb.c3 = (cell3 *)malloc(sizeof(cell3));
        else jb.c2 = (cell2 *)malloc(sizeof(cell2));
        int *ford = (int *)malloc(sizeof(int) * OR_MAXF);
#pragma omp for schedule(dynamic, 64)
        for (long long ci = 0; ci < ncell; ci++) {
            long long i = cells ? cells[ci] : ci;
            jb.self = i;
            for (int a = 0; a < 3; a++) jb.p[a] = a < dim ? pos[i * dim + a] : 0.0;
            jb.rp = radii ? radii[i] : 0.0;
            int st;
            if (method == 1) {
                int bp[3] = {0, 0, 0};
                for (int a = 0; a < dim; a++) {
                    int b = (int)floor((jb.p[a] - lo[a]) / cx.h[a]);
                    if (b < 0) b = 0;
                    if (b >= cx.nb[a]) b = cx.nb[a] - 1;
                    bp[a] = b;
                }
                st = cell_grid(&cx, &jb, bp);
            } else {
                st = cell_brute(&cx, &jb);
            }
            stats_t S;
            memset(&S, 0, sizeof S);
            int nfaces = 0;
            if (st == ST_OK) {
                if (dim == 3) { stats3(jb.c3, merge_rel * cx.s, &S, ford); nfaces = jb.c3->nf; }
                else { stats2(jb.c2, &S); nfaces = jb.c2->nv; }
                if (nfaces > maxf) { st = ST_CAP; nfaces = 0; memset(&S, 0, sizeof S); }
            }
            vol[ci] = S.vol;
            area[ci] = S.area;
            for (int a = 0; a < dim; a++) cen[ci * dim + a] = S.cen[a];
            nv[ci] = S.nv; ne[ci] = S.ne; nf[ci] = S.nf;
            status[ci] = st;
            if (rmax) rmax[ci] = S.R;
            if (ntested) ntested[ci] = jb.ntested;
            if (ncut) ncut[ci] = jb.ncut;
            if (wlen) { wlen[ci] = S.wlen; whash[ci] = S.whash; wsym[ci] = S.wsym; }
            /* faces in canonical order: ascending (id, image shift) */
            long long *oid = nbr_id + ci * maxf;
            int *oim = nbr_img + ci * maxf * 3, *oor = face_order + ci * maxf;
            for (int u = 0; u < nfaces; u++) {
                long long id; const int *im; int ordv;
                if (dim == 3) { id = jb.c3->f[u].id; im = jb.c3->f[u].img; ordv = ford[u]; }
                else { id = jb.c2->lid[u]; im = jb.c2->limg[u]; ordv = 2; }
                int w = u;
                /* insertion into the sorted prefix */
                while (w > 0) {
                    long long pid = oid[w - 1];
                    const int *pim = &oim[(w - 1) * 3];
                    int gt = pid > id;
                    if (pid == id) {
                        for (int a = 0; a < 3; a++) {
                            int ia = a < dim ? im[a] : 0;
                            if (pim[a] != ia) { gt = pim[a] > ia; break; }
                        }
                    }
                    if (!gt) break;
                    oid[w] = oid[w - 1];
                    oim[w * 3] = oim[(w - 1) * 3]; oim[w * 3 + 1] = oim[(w - 1) * 3 + 1]; oim[w * 3 + 2] = oim[(w - 1) * 3 + 2];
                    oor[w] = oor[w - 1];
                    w--;
                }
                oid[w] = id;
                for (int a = 0; a < 3; a++) oim[w * 3 + a] = a < dim ? im[a] : 0;
                oor[w] = ordv;
            }
        }
        free(jb.c3); free(jb.c2); free(ford);
    }
    free(cx.bstart);
    free(cx.bidx);
    return 0;
}

/* Grid dimensions from the target particles per block (Sec. 2.1.4):
 * lambda = (N / (n_opt * volume))^(1/dim), n_a = round_mode(lambda * L_a),
 * never below 1.  round_mode 0 is the ceiling the text states, 1 the floor
 * that reproduces Table 3. */
void vo_grid_size(int dim, long long n, const double *lo, const double *hi, double n_opt,
                  int round_mode, int *out) {
    double V = 1;
    for (int a = 0; a < dim; a++) V *= hi[a] - lo[a];
    double lam = pow((double)n / (n_opt * V), 1.0 / dim);
    for (int a = 0; a < dim; a++) {
        double x = lam * (hi[a] - lo[a]);
        int v = round_mode ? (int)floor(x) : (int)ceil(x);
        out[a] = v < 1 ? 1 : v;
    }
}
