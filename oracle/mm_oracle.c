/* mm_oracle.c -- plain, slow FP64 CPU oracle of the moving-mesh hot path.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg may call it; the product path never does.  It shares no
 * code with the CUDA library and favours obviousness over speed:
 *   - a cell is a list of face polygons clipped one bisector plane at a time
 *     (Sutherland-Hodgman per face), in increasing distance order, stopping
 *     once the next generator is more than twice as far as the farthest
 *     vertex (Sec. 3);
 *   - volumes and centroids come from tetrahedra about the generator, face
 *     areas from triangle fans about the vertex mean;
 *   - the hydro loops run over unique faces and scatter to both cells;
 *   - the half-step uses the explicit Euler flux Jacobians A_d (Sec. 4.1);
 *   - the Riemann problem is rotated into an explicit (n, t1, t2) basis (Sec. 4).
 *
 * Where the paper is silent or garbled it is read as: the centroid
 * Green-Gauss gradient M g = b; the S10 limiter over neighbour centroids; the
 * Duffell-MacFadyen factor clamped at 0 and counted only where Delta is
 * nonzero beyond rounding; Davis wave speeds; the outward-flux sign of the
 * update; floors on rho and eps; the entropy column as a passive scalar
 * upwind of the contact, switched at the volume the faces sweep the cell to.
 *
 * Pins (CPU tests): closed-form lattice cells, Qhull's Voronoi diagram of the
 * unrolled box, Toro's exact star states and the HLLC jump conditions, the
 * one-dimensional scheme on planar lattices, the geometric conservation law,
 * and the step's symmetries.
 */
#include "mm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static int shift_code(const int *s) { return (s[0] + 1) + 3 * (s[1] + 1) + 9 * (s[2] + 1); }

/* ------------------------------------------------------------------------ */
/* Polyhedron as a list of convex face polygons (Sec. 3)                     */
/* ------------------------------------------------------------------------ */
#define OMAXF 192
#define OMAXV 64

typedef struct {
    int nf;
    int nb[OMAXF];
    int sh[OMAXF][3];
    double q[OMAXF][3]; /* plane: x . q <= off, q = relative position of the neighbour */
    double off[OMAXF];
    int nv[OMAXF];
    double v[OMAXF][OMAXV][3];
} opoly;

/* The starting cell is the box [-L/2, L/2] centred on the generator: its six
 * planes are the bisectors with the generator's own periodic images, so the
 * true cell always lies inside it. */
static void poly_init_box(opoly *P, const double *box, int self)
{
    const double hx = 0.5 * box[0], hy = 0.5 * box[1], hz = 0.5 * box[2];
    P->nf = 6;
    for (int f = 0; f < 6; ++f) {
        int d = f / 2, sg = (f % 2 == 0) ? 1 : -1;
        P->nb[f] = self;
        P->sh[f][0] = P->sh[f][1] = P->sh[f][2] = 0;
        P->sh[f][d] = sg;
        P->q[f][0] = P->q[f][1] = P->q[f][2] = 0.0;
        P->q[f][d] = sg * box[d];
        P->off[f] = 0.5 * box[d] * box[d];
        P->nv[f] = 4;
        /* four corners of the face, in cyclic order */
        static const int uv[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
        double h[3] = {hx, hy, hz};
        int a = (d + 1) % 3, b = (d + 2) % 3;
        for (int k = 0; k < 4; ++k) {
            P->v[f][k][d] = sg * h[d];
            P->v[f][k][a] = uv[k][0] * h[a];
            P->v[f][k][b] = uv[k][1] * h[b];
        }
    }
}

static double poly_rmax2(const opoly *P)
{
    double r = 0.0;
    for (int f = 0; f < P->nf; ++f)
        for (int k = 0; k < P->nv[f]; ++k) {
            double d = dot3(P->v[f][k], P->v[f][k]);
            if (d > r) r = d;
        }
    return r;
}

typedef struct { double ang; double p[3]; } angpt;
static int cmp_ang(const void *a, const void *b)
{
    double x = ((const angpt *)a)->ang, y = ((const angpt *)b)->ang;
    return (x > y) - (x < y);
}

/* Clip the cell by the half-space x.q <= off.  Returns 1 if the plane cut the
 * cell (a new face was added), 0 if it missed, -1 on a capacity overflow. */
static int poly_clip(opoly *P, const double *q, double off, int nb, const int *sh)
{
    int any = 0;
    for (int f = 0; f < P->nf && !any; ++f)
        for (int k = 0; k < P->nv[f]; ++k)
            if (dot3(q, P->v[f][k]) - off > 0.0) { any = 1; break; }
    if (!any) return 0;

    static double newp[2 * OMAXF * 2][3];
    int nnew = 0;
    int keep = 0;
    for (int f = 0; f < P->nf; ++f) {
        int nv = P->nv[f];
        double s[OMAXV];
        int nout = 0;
        for (int k = 0; k < nv; ++k) {
            s[k] = dot3(q, P->v[f][k]) - off;
            if (s[k] > 0.0) ++nout;
        }
        if (nout == nv) continue; /* face entirely beyond the plane: dropped */
        double out[OMAXV + 2][3];
        int no = 0;
        if (nout == 0) {
            for (int k = 0; k < nv; ++k) {
                memcpy(out[no++], P->v[f][k], sizeof(double) * 3);
                if (s[k] == 0.0 && nnew < 4 * OMAXF) memcpy(newp[nnew++], P->v[f][k], sizeof(double) * 3);
            }
        } else {
            for (int k = 0; k < nv; ++k) {
                int k2 = (k + 1) % nv;
                const double *a = P->v[f][k], *b = P->v[f][k2];
                double sa = s[k], sb = s[k2];
                if (sa <= 0.0) {
                    if (no >= OMAXV) return -1;
                    memcpy(out[no++], a, sizeof(double) * 3);
                    if (sa == 0.0 && nnew < 4 * OMAXF) memcpy(newp[nnew++], a, sizeof(double) * 3);
                }
                if ((sa < 0.0 && sb > 0.0) || (sa > 0.0 && sb < 0.0)) {
                    double t = sa / (sa - sb);
                    double p[3] = {a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]), a[2] + t * (b[2] - a[2])};
                    if (no >= OMAXV) return -1;
                    memcpy(out[no++], p, sizeof(double) * 3);
                    if (nnew < 4 * OMAXF) memcpy(newp[nnew++], p, sizeof(double) * 3);
                }
            }
        }
        if (no < 3) continue;
        /* keep face f (compact to slot keep) */
        P->nb[keep] = P->nb[f];
        memcpy(P->sh[keep], P->sh[f], sizeof(int) * 3);
        memcpy(P->q[keep], P->q[f], sizeof(double) * 3);
        P->off[keep] = P->off[f];
        P->nv[keep] = no;
        memcpy(P->v[keep], out, sizeof(double) * 3 * no);
        ++keep;
    }
    P->nf = keep;

    /* the new face: distinct intersection points ordered by angle */
    double scale = sqrt(dot3(q, q));
    double tol = 1e-13 * scale;
    int nd = 0;
    static angpt pts[4 * OMAXF];
    for (int k = 0; k < nnew; ++k) {
        int dup = 0;
        for (int m = 0; m < nd; ++m) {
            double dx = pts[m].p[0] - newp[k][0], dy = pts[m].p[1] - newp[k][1], dz = pts[m].p[2] - newp[k][2];
            if (sqrt(dx * dx + dy * dy + dz * dz) <= tol) { dup = 1; break; }
        }
        if (!dup) { memcpy(pts[nd].p, newp[k], sizeof(double) * 3); ++nd; }
    }
    if (nd < 3) return 1;
    if (nd > OMAXV || P->nf >= OMAXF) return -1;
    double m[3] = {0, 0, 0};
    for (int k = 0; k < nd; ++k) for (int d = 0; d < 3; ++d) m[d] += pts[k].p[d];
    for (int d = 0; d < 3; ++d) m[d] /= nd;
    double nrm[3] = {q[0] / scale, q[1] / scale, q[2] / scale};
    double ax[3] = {1, 0, 0};
    if (fabs(nrm[0]) > 0.8) { ax[0] = 0; ax[1] = 1; }
    double e1[3], e2[3];
    cross3(nrm, ax, e1);
    double l1 = sqrt(dot3(e1, e1));
    for (int d = 0; d < 3; ++d) e1[d] /= l1;
    cross3(nrm, e1, e2);
    for (int k = 0; k < nd; ++k) {
        double r[3] = {pts[k].p[0] - m[0], pts[k].p[1] - m[1], pts[k].p[2] - m[2]};
        pts[k].ang = atan2(dot3(r, e2), dot3(r, e1));
    }
    qsort(pts, nd, sizeof(angpt), cmp_ang);
    int f = P->nf++;
    P->nb[f] = nb;
    memcpy(P->sh[f], sh, sizeof(int) * 3);
    memcpy(P->q[f], q, sizeof(double) * 3);
    P->off[f] = off;
    P->nv[f] = nd;
    for (int k = 0; k < nd; ++k) memcpy(P->v[f][k], pts[k].p, sizeof(double) * 3);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Candidates                                                                */
/* ------------------------------------------------------------------------ */
typedef struct { double d2; int j; int code; double q[3]; int sh[3]; } ocand;

static int cmp_cand(const void *a, const void *b)
{
    const ocand *x = (const ocand *)a, *y = (const ocand *)b;
    if (x->d2 != y->d2) return (x->d2 > y->d2) - (x->d2 < y->d2);
    if (x->j != y->j) return (x->j > y->j) - (x->j < y->j);
    return (x->code > y->code) - (x->code < y->code);
}

/* A generator's own images across the six box faces are the starting planes. */
static int is_axis_self(int i, int j, const int *s)
{
    if (i != j) return 0;
    int nz = (s[0] != 0) + (s[1] != 0) + (s[2] != 0);
    return nz == 1;
}

typedef struct {
    ocand *c;
    int64_t n, cap;
} cand_list;

static int cand_push(cand_list *L, const ocand *c)
{
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 256;
        ocand *p = (ocand *)realloc(L->c, sizeof(ocand) * nc);
        if (!p) return -1;
        L->c = p;
        L->cap = nc;
    }
    L->c[L->n++] = *c;
    return 0;
}

/* Clip by the sorted candidates c[0..m) until the next one is more than twice
 * as far as the farthest vertex.  Returns -1 on overflow, else the index of
 * the first unprocessed candidate. */
static int64_t clip_sorted(opoly *P, const ocand *c, int64_t m, double *rmax2)
{
    int64_t k = 0;
    for (; k < m; ++k) {
        if (c[k].d2 > 4.0 * (*rmax2)) break;
        int r = poly_clip(P, c[k].q, 0.5 * c[k].d2, c[k].j, c[k].sh);
        if (r < 0) return -1;
        if (r > 0) *rmax2 = poly_rmax2(P);
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Face and cell geometry                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double vol, cen[3];
    int nf;
    int nb[OMAXF], sh[OMAXF][3];
    double area[OMAXF], nrm[OMAXF][3], fc[OMAXF][3];
} ogeom;

static void poly_geometry(const opoly *P, ogeom *G)
{
    G->vol = 0.0;
    G->cen[0] = G->cen[1] = G->cen[2] = 0.0;
    G->nf = 0;
    for (int f = 0; f < P->nf; ++f) {
        int nv = P->nv[f];
        double m[3] = {0, 0, 0};
        for (int k = 0; k < nv; ++k) for (int d = 0; d < 3; ++d) m[d] += P->v[f][k][d];
        for (int d = 0; d < 3; ++d) m[d] /= nv;
        double area = 0.0, fc[3] = {0, 0, 0};
        for (int k = 0; k < nv; ++k) {
            const double *a = P->v[f][k], *b = P->v[f][(k + 1) % nv];
            double ea[3] = {a[0] - m[0], a[1] - m[1], a[2] - m[2]};
            double eb[3] = {b[0] - m[0], b[1] - m[1], b[2] - m[2]};
            double c[3];
            cross3(ea, eb, c);
            double at = 0.5 * sqrt(dot3(c, c));
            area += at;
            for (int d = 0; d < 3; ++d) fc[d] += at * (m[d] + a[d] + b[d]) / 3.0;
            /* tetrahedron (generator, m, a, b) */
            double mc[3];
            cross3(a, b, mc);
            double vt = fabs(dot3(m, mc)) / 6.0;
            G->vol += vt;
            for (int d = 0; d < 3; ++d) G->cen[d] += vt * (m[d] + a[d] + b[d]) / 4.0;
        }
        int g = G->nf++;
        G->nb[g] = P->nb[f];
        memcpy(G->sh[g], P->sh[f], sizeof(int) * 3);
        G->area[g] = area;
        double ql = sqrt(dot3(P->q[f], P->q[f]));
        for (int d = 0; d < 3; ++d) {
            G->nrm[g][d] = P->q[f][d] / ql;
            G->fc[g][d] = area > 0.0 ? fc[d] / area : m[d];
        }
    }
    for (int d = 0; d < 3; ++d) G->cen[d] /= G->vol;
}

/* ------------------------------------------------------------------------ */
/* Tessellation drivers                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const double *pos;
    double box[3];
    int g[3];
    double bs[3];
    int64_t *start; /* [nbins+1] */
    int64_t *items; /* [n] */
} ogrid;

static void grid_build(ogrid *G, int64_t n, const double *pos, const double *box)
{
    G->n = n;
    G->pos = pos;
    double s = cbrt(box[0] * box[1] * box[2] / (double)n);
    int64_t nb = 1;
    for (int d = 0; d < 3; ++d) {
        G->box[d] = box[d];
        int g = (int)floor(box[d] / s);
        if (g < 1) g = 1;
        G->g[d] = g;
        G->bs[d] = box[d] / g;
        nb *= g;
    }
    G->start = (int64_t *)calloc(nb + 1, sizeof(int64_t));
    G->items = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int64_t *bin = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = 0, mul = 1;
        for (int d = 0; d < 3; ++d) {
            int c = (int)floor(pos[3 * i + d] / G->bs[d]);
            if (c >= G->g[d]) c = G->g[d] - 1;
            if (c < 0) c = 0;
            b += mul * c;
            mul *= G->g[d];
        }
        bin[i] = b;
        G->start[b + 1]++;
    }
    for (int64_t b = 0; b < nb; ++b) G->start[b + 1] += G->start[b];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * nb);
    memcpy(cur, G->start, sizeof(int64_t) * nb);
    for (int64_t i = 0; i < n; ++i) G->items[cur[bin[i]]++] = i;
    free(cur);
    free(bin);
}

static void grid_free(ogrid *G)
{
    free(G->start);
    free(G->items);
}

static void make_cand(int64_t i, int64_t j, const int *s, const double *pos, const double *box, ocand *c)
{
    c->j = (int)j;
    memcpy(c->sh, s, sizeof(int) * 3);
    c->code = shift_code(s);
    for (int d = 0; d < 3; ++d) c->q[d] = pos[3 * j + d] + s[d] * box[d] - pos[3 * i + d];
    c->d2 = dot3(c->q, c->q);
}

/* Brute force: all generators and their 27 images (offsets with a component
 * of magnitude 2 or more can never cut when positions lie in [0, L)).  Only
 * candidates closer than tau are sorted; tau grows to 2 r_max when the sorted
 * batch runs out before the stopping test passes, which keeps the global
 * processing order exactly the sorted order. */
static int cell_bruteforce(int64_t i, int64_t n, const double *pos, const double *box, opoly *P,
                           cand_list *L)
{
    poly_init_box(P, box, (int)i);
    double rmax2 = poly_rmax2(P);
    double tau = 0.0, s = cbrt(box[0] * box[1] * box[2] / (double)n);
    double tau_next = 16.0 * s * s;
    for (;;) {
        L->n = 0;
        for (int64_t j = 0; j < n; ++j)
            for (int sz = -1; sz <= 1; ++sz)
                for (int sy = -1; sy <= 1; ++sy)
                    for (int sx = -1; sx <= 1; ++sx) {
                        int sh[3] = {sx, sy, sz};
                        if (j == i && sx == 0 && sy == 0 && sz == 0) continue;
                        if (is_axis_self((int)i, (int)j, sh)) continue;
                        ocand c;
                        make_cand(i, j, sh, pos, box, &c);
                        if (c.d2 >= tau && c.d2 < tau_next && c.d2 <= 4.0 * rmax2)
                            if (cand_push(L, &c)) return 3;
                    }
        qsort(L->c, L->n, sizeof(ocand), cmp_cand);
        int64_t k = clip_sorted(P, L->c, L->n, &rmax2);
        if (k < 0) return 3;
        if (k < L->n) return 0;              /* stopped inside the batch */
        if (4.0 * rmax2 < tau_next) return 0; /* nothing closer than 2 r_max remains */
        tau = tau_next;
        tau_next = 4.0 * rmax2 * (1.0 + 1e-12) + 1e-300;
        if (tau_next <= tau) return 0;
    }
}

/* Grid mode: gather the (2r+1)^3 block of bins around the generator's bin,
 * clip from scratch in sorted order, and accept once 2 r_max is inside the
 * guaranteed radius of the block; otherwise grow r and start over. */
static int cell_grid(int64_t i, const ogrid *G, opoly *P, cand_list *L)
{
    const double *pos = G->pos;
    int cb[3];
    for (int d = 0; d < 3; ++d) {
        int c = (int)floor(pos[3 * i + d] / G->bs[d]);
        if (c >= G->g[d]) c = G->g[d] - 1;
        if (c < 0) c = 0;
        cb[d] = c;
    }
    for (int r = 1; r < 1000; ++r) {
        L->n = 0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    int off[3] = {dx, dy, dz}, bb[3], sh[3];
                    for (int d = 0; d < 3; ++d) {
                        int c = cb[d] + off[d];
                        int s = (int)floor((double)c / G->g[d]);
                        bb[d] = c - s * G->g[d];
                        sh[d] = s;
                    }
                    int64_t b = bb[0] + (int64_t)G->g[0] * (bb[1] + (int64_t)G->g[1] * bb[2]);
                    for (int64_t t = G->start[b]; t < G->start[b + 1]; ++t) {
                        int64_t j = G->items[t];
                        if (j == i && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
                        if (is_axis_self((int)i, (int)j, sh)) continue;
                        ocand c;
                        make_cand(i, j, sh, pos, G->box, &c);
                        if (cand_push(L, &c)) return 3;
                    }
                }
        qsort(L->c, L->n, sizeof(ocand), cmp_cand);
        poly_init_box(P, G->box, (int)i);
        double rmax2 = poly_rmax2(P);
        /* guaranteed radius: distance from the generator to the block boundary */
        double R = 1e300;
        for (int d = 0; d < 3; ++d) {
            double lo = (cb[d] - r) * G->bs[d], hi = (cb[d] + r + 1) * G->bs[d];
            double x = pos[3 * i + d];
            if (x - lo < R) R = x - lo;
            if (hi - x < R) R = hi - x;
        }
        /* only candidates inside the guaranteed radius are complete */
        int64_t m = 0;
        while (m < L->n && L->c[m].d2 < R * R) ++m;
        int64_t k = clip_sorted(P, L->c, m, &rmax2);
        if (k < 0) return 3;
        if (4.0 * rmax2 <= R * R) return 0;
    }
    return 3;
}

static int emit_cell(int64_t i, const double *pos, const opoly *P, double area_min,
                     double *volume, double *centroid, int64_t cap, int64_t *nface,
                     int32_t *f_cell, int32_t *f_nb, int32_t *f_shift, double *f_area,
                     double *f_normal, double *f_centroid, ogeom *G)
{
    poly_geometry(P, G);
    volume[i] = G->vol;
    for (int d = 0; d < 3; ++d) centroid[3 * i + d] = pos[3 * i + d] + G->cen[d];
    double thr = area_min;
    for (int f = 0; f < G->nf; ++f) {
        if (!(G->area[f] > thr)) continue;
        int64_t k = (*nface)++;
        if (k >= cap) return 1;
        f_cell[k] = (int32_t)i;
        f_nb[k] = G->nb[f];
        for (int d = 0; d < 3; ++d) {
            f_shift[3 * k + d] = G->sh[f][d];
            f_normal[3 * k + d] = G->nrm[f][d];
            f_centroid[3 * k + d] = pos[3 * i + d] + G->fc[f][d];
        }
        f_area[k] = G->area[f];
    }
    return 0;
}

/* Tie rule for near-degenerate contacts: a face is kept when its area exceeds
 * area_rel times the mean cell area scale (V_box / n)^(2/3).  The threshold is
 * one number for the whole box, so both cells of a face take the same
 * decision. */
static double face_area_min(int64_t n, const double *box, double area_rel)
{
    return area_rel * pow(box[0] * box[1] * box[2] / (double)n, 2.0 / 3.0);
}

static int check_input(int64_t n, const double *pos, const double *box)
{
    if (n <= 0) return 2;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0.0) || !isfinite(box[d])) return 2;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d)
            if (!(pos[3 * i + d] >= 0.0 && pos[3 * i + d] < box[d])) return 2;
    return 0;
}

int orc_tessellate(int64_t n, const double *pos, const double *box, int mode, double area_rel,
                   double *volume, double *centroid, int64_t cap, int64_t *nface,
                   int32_t *f_cell, int32_t *f_nb, int32_t *f_shift, double *f_area,
                   double *f_normal, double *f_centroid)
{
    *nface = 0;
    if (check_input(n, pos, box)) return 2;
    opoly *P = (opoly *)malloc(sizeof(opoly));
    ogeom *G = (ogeom *)malloc(sizeof(ogeom));
    cand_list L = {0, 0, 0};
    ogrid grid;
    double amin = face_area_min(n, box, area_rel);
    if (mode == 1) grid_build(&grid, n, pos, box);
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; ++i) {
        rc = (mode == 1) ? cell_grid(i, &grid, P, &L) : cell_bruteforce(i, n, pos, box, P, &L);
        if (rc == 0)
            rc = emit_cell(i, pos, P, amin, volume, centroid, cap, nface, f_cell, f_nb, f_shift,
                           f_area, f_normal, f_centroid, G);
    }
    if (mode == 1) grid_free(&grid);
    free(L.c);
    free(P);
    free(G);
    return rc;
}

int orc_tessellate_subset(int64_t n, const double *pos, const double *box, double area_rel,
                          int64_t m, const int64_t *cells, double *volume, double *centroid,
                          int64_t cap, int64_t *nface, int32_t *f_cell, int32_t *f_nb,
                          int32_t *f_shift, double *f_area, double *f_normal, double *f_centroid)
{
    *nface = 0;
    if (check_input(n, pos, box)) return 2;
    opoly *P = (opoly *)malloc(sizeof(opoly));
    ogeom *G = (ogeom *)malloc(sizeof(ogeom));
    cand_list L = {0, 0, 0};
    ogrid grid;
    double amin = face_area_min(n, box, area_rel);
    grid_build(&grid, n, pos, box);
    int rc = 0;
    for (int64_t t = 0; t < m && rc == 0; ++t) {
        int64_t i = cells[t];
        if (i < 0 || i >= n) { rc = 2; break; }
        rc = cell_grid(i, &grid, P, &L);
        if (rc == 0)
            rc = emit_cell(i, pos, P, amin, volume, centroid, cap, nface, f_cell, f_nb, f_shift,
                           f_area, f_normal, f_centroid, G);
    }
    grid_free(&grid);
    free(L.c);
    free(P);
    free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Equation of state and floors (Sec. 4, 4.1, 6)                             */
/* ------------------------------------------------------------------------ */
/* Floors on density and specific internal energy, applied to a per-volume
 * state (rho, m, E).  Below the density floor the state carries no usable
 * velocity (it may even be negative after reconstruction), so it is reset to
 * the floor density at rest with the floor internal energy.  Otherwise only
 * the internal energy is raised to rho * eps_floor if needed, keeping rho and
 * m; an untouched state is returned bit for bit. */
void orc_floor_state(const double *W, const orc_cfg *cfg, double *Wout, int *changed)
{
    int ch = 0;
    if (!(W[0] >= cfg->rho_floor)) {
        Wout[0] = cfg->rho_floor;
        Wout[1] = Wout[2] = Wout[3] = 0.0;
        Wout[4] = cfg->rho_floor * cfg->eps_floor;
        if (changed) *changed = 1;
        return;
    }
    double rho = W[0];
    double m2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
    double ke = 0.5 * m2 / rho;
    double E = W[4];
    if (!(E - ke >= rho * cfg->eps_floor)) { E = rho * cfg->eps_floor + ke; ch = 1; }
    Wout[0] = rho;
    Wout[1] = W[1];
    Wout[2] = W[2];
    Wout[3] = W[3];
    Wout[4] = E;
    if (changed) *changed = ch;
}

/* Physical flux along a unit direction: (rho u_n, m u_n + P n, (E + P) u_n). */
void orc_euler_flux(const double *W, const double *nrm, double gamma, double *F)
{
    double rho = W[0];
    double v[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    double P = (gamma - 1.0) * (W[4] - 0.5 * rho * dot3(v, v));
    double un = dot3(v, nrm);
    F[0] = rho * un;
    for (int k = 0; k < 3; ++k) F[1 + k] = W[1 + k] * un + P * nrm[k];
    F[4] = (W[4] + P) * un;
}

/* Jacobian A_d = dF_d/dW of the Euler flux along axis d, written out from
 * F_d = (m_d, m_k m_d / rho + P delta_kd, (E + P) m_d / rho). */
void orc_flux_jacobian(const double *W, int d, double gamma, double *A)
{
    double rho = W[0];
    double u[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    double q2 = dot3(u, u);
    double g1 = gamma - 1.0;
    double P = g1 * (W[4] - 0.5 * rho * q2);
    double H = (W[4] + P) / rho;
    memset(A, 0, sizeof(double) * 25);
    /* mass row */
    A[0 * 5 + 1 + d] = 1.0;
    /* momentum rows */
    for (int k = 0; k < 3; ++k) {
        double *row = A + (1 + k) * 5;
        row[0] = -u[k] * u[d] + (k == d ? 0.5 * g1 * q2 : 0.0);
        for (int l = 0; l < 3; ++l)
            row[1 + l] = (k == l ? u[d] : 0.0) + (d == l ? u[k] : 0.0) - (k == d ? g1 * u[l] : 0.0);
        row[4] = (k == d) ? g1 : 0.0;
    }
    /* energy row */
    double *row = A + 4 * 5;
    row[0] = u[d] * (0.5 * g1 * q2 - H);
    for (int l = 0; l < 3; ++l) row[1 + l] = -g1 * u[l] * u[d] + (d == l ? H : 0.0);
    row[4] = gamma * u[d];
}

/* ------------------------------------------------------------------------ */
/* Gradients and limiters (Sec. 4.1)                                         */
/* ------------------------------------------------------------------------ */
static void face_delta(const double *centroid, const double *box, int32_t i, int32_t j, const int32_t *sh,
                       double *d)
{
    for (int a = 0; a < 3; ++a) d[a] = centroid[3 * j + a] + sh[a] * box[a] - centroid[3 * i + a];
}

/* 3x3 solve by Gaussian elimination with partial pivoting (nc <= 6 rhs columns). */
static void solve3(const double *M, const double *B /* [3][nc] */, int nc, double *X /* [3][nc] */)
{
    double a[3][9];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) a[r][c] = M[3 * r + c];
        for (int c = 0; c < nc; ++c) a[r][3 + c] = B[nc * r + c];
    }
    for (int c = 0; c < 3; ++c) {
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
        if (p != c)
            for (int k = 0; k < 3 + nc; ++k) { double t = a[c][k]; a[c][k] = a[p][k]; a[p][k] = t; }
        for (int r = c + 1; r < 3; ++r) {
            double f = a[r][c] / a[c][c];
            for (int k = c; k < 3 + nc; ++k) a[r][k] -= f * a[c][k];
        }
    }
    for (int c = 0; c < nc; ++c)
        for (int r = 2; r >= 0; --r) {
            double s = a[r][3 + c];
            for (int k = r + 1; k < 3; ++k) s -= a[r][k] * X[nc * k + c];
            X[nc * r + c] = s / a[r][r];
        }
}

static int state_width(const orc_cfg *cfg) { return cfg->entropy ? 6 : 5; }

/* Cell-centred Green-Gauss gradient: with d_ij the vector between the two
 * cell centroids across face ij (image-corrected), M_i = 1/2 sum A n (x) d and
 * b_i = 1/2 sum A (W_j - W_i) n, and grad W_i = M_i^{-1} b_i, exact for
 * linear fields.  Then the S10 factor min(1, psi_ij) over the neighbours
 * (psi from the neighbourhood max/min and Delta_ij = grad . (c_j - c_i)), and
 * optionally the Duffell-MacFadyen factor min(1, max(0, theta (W_j - W_i) /
 * Delta_ij)) over the neighbours whose Delta_ij is nonzero beyond rounding.  limiter 3 is S10 with Delta_ij measured to the face centroid,
 * grad . (x_f - c_i), as in the original S10 scheme.  Every state column,
 * the entropy column included, is treated alike (Sec. 4.3). */
void orc_gradient(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const int32_t *fshift,
                  const double *farea, const double *fnormal, const double *fcentroid, const double *centroid,
                  const double *box, const double *W, const orc_cfg *cfg, double *grad)
{
    const int ng = state_width(cfg);
    double *M = (double *)calloc(9 * n, sizeof(double));
    double *B = (double *)calloc(3 * ng * n, sizeof(double)); /* [n][3][ng] */
    double *wmax = (double *)malloc(sizeof(double) * ng * n);
    double *wmin = (double *)malloc(sizeof(double) * ng * n);
    double *psi = (double *)malloc(sizeof(double) * ng * n);
    double *psidm = (double *)malloc(sizeof(double) * ng * n);
    memcpy(wmax, W, sizeof(double) * ng * n);
    memcpy(wmin, W, sizeof(double) * ng * n);
    for (int64_t f = 0; f < nf; ++f) {
        int32_t i = fi[f], j = fj[f];
        double d[3];
        face_delta(centroid, box, i, j, fshift + 3 * f, d);
        const double *nr = fnormal + 3 * f;
        double A = farea[f];
        /* cell i sees (n, d); cell j sees (-n, -d): both products are equal */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double v = 0.5 * A * nr[a] * d[b];
                M[9 * i + 3 * a + b] += v;
                M[9 * j + 3 * a + b] += v;
            }
        for (int k = 0; k < ng; ++k) {
            double dw = W[ng * j + k] - W[ng * i + k];
            for (int a = 0; a < 3; ++a) {
                B[3 * ng * i + ng * a + k] += 0.5 * A * dw * nr[a];
                B[3 * ng * j + ng * a + k] += 0.5 * A * dw * nr[a];
            }
            if (W[ng * j + k] > wmax[ng * i + k]) wmax[ng * i + k] = W[ng * j + k];
            if (W[ng * j + k] < wmin[ng * i + k]) wmin[ng * i + k] = W[ng * j + k];
            if (W[ng * i + k] > wmax[ng * j + k]) wmax[ng * j + k] = W[ng * i + k];
            if (W[ng * i + k] < wmin[ng * j + k]) wmin[ng * j + k] = W[ng * i + k];
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double X[18];
        solve3(M + 9 * i, B + 3 * ng * i, ng, X);
        for (int k = 0; k < ng; ++k)
            for (int a = 0; a < 3; ++a) grad[3 * ng * i + 3 * k + a] = X[ng * a + k];
    }
    for (int64_t t = 0; t < ng * n; ++t) psi[t] = psidm[t] = 1.0;
    if (cfg->limiter >= 1) {
        for (int64_t f = 0; f < nf; ++f) {
            int32_t i = fi[f], j = fj[f];
            double d[3];
            face_delta(centroid, box, i, j, fshift + 3 * f, d);
            for (int side = 0; side < 2; ++side) {
                int32_t c = side ? j : i, o = side ? i : j;
                double sg = side ? -1.0 : 1.0;
                double dv[3];
                for (int a = 0; a < 3; ++a) {
                    if (cfg->limiter == 3) {
                        /* face centroid in this cell's frame minus the cell centroid */
                        double xf = fcentroid[3 * f + a] - (side ? fshift[3 * f + a] * box[a] : 0.0);
                        dv[a] = xf - centroid[3 * c + a];
                    } else {
                        dv[a] = sg * d[a];
                    }
                }
                for (int k = 0; k < ng; ++k) {
                    const double *g = grad + 3 * ng * c + 3 * k;
                    double del = g[0] * dv[0] + g[1] * dv[1] + g[2] * dv[2];
                    double p = 1.0;
                    if (del > 0.0) p = (wmax[ng * c + k] - W[ng * c + k]) / del;
                    else if (del < 0.0) p = (wmin[ng * c + k] - W[ng * c + k]) / del;
                    if (p < psi[ng * c + k]) psi[ng * c + k] = p;
                    /* the Duffell-MacFadyen ratio counts only where Delta is
                     * nonzero (Sec. 4.1); a Delta within 2^-40 |g|_1 |d|_1 (well
                     * above the ~1e-15 of it that the rounding of the gradient and
                     * the centroids leaves, far below any Delta that matters) is
                     * zero in exact arithmetic: a gradient orthogonal to d, as
                     * toward the equal-valued transverse neighbours of a lattice
                     * or across a row of symmetry; it does not count */
                    if (cfg->limiter == 2) {
                        double gd = (fabs(g[0]) + fabs(g[1]) + fabs(g[2])) * (fabs(dv[0]) + fabs(dv[1]) + fabs(dv[2]));
                        if (fabs(del) > 0x1p-40 * gd) {
                            double pd = cfg->theta * (W[ng * o + k] - W[ng * c + k]) / del;
                            if (pd < 0.0) pd = 0.0;
                            if (pd < psidm[ng * c + k]) psidm[ng * c + k] = pd;
                        }
                    }
                }
            }
        }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < ng; ++k) {
                double alpha = psi[ng * i + k] < 1.0 ? psi[ng * i + k] : 1.0;
                if (cfg->limiter == 2) alpha *= (psidm[ng * i + k] < 1.0 ? psidm[ng * i + k] : 1.0);
                for (int a = 0; a < 3; ++a) grad[3 * ng * i + 3 * k + a] *= alpha;
            }
    }
    free(M);
    free(B);
    free(wmax);
    free(wmin);
    free(psi);
    free(psidm);
}

/* Half-step predictor: dW/dt = -sum_d A_d(W) dW/dx_d, Wh = W + dt/2 dW/dt.
 * The entropy column's flux is (rho A) m_d / rho, so its Jacobian row along
 * d is (-A u_d, A delta_{ld}, 0, u_d) in (rho, m_l, E, rho A). */
void orc_half_step(int64_t n, const double *W, const double *grad, const orc_cfg *cfg, double dt,
                   double *Wh)
{
    const int ng = state_width(cfg);
    for (int64_t i = 0; i < n; ++i) {
        const double *Wi = W + ng * i;
        const double *g = grad + 3 * ng * i;
        double rate[6] = {0, 0, 0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            double A[25];
            orc_flux_jacobian(Wi, d, cfg->gamma, A);
            for (int r = 0; r < 5; ++r)
                for (int c = 0; c < 5; ++c) rate[r] -= A[5 * r + c] * g[3 * c + d];
            if (ng == 6) {
                double a = Wi[5] / Wi[0], ud = Wi[1 + d] / Wi[0];
                rate[5] -= -a * ud * g[d] + a * g[3 * (1 + d) + d] + ud * g[15 + d];
            }
        }
        for (int r = 0; r < ng; ++r) Wh[ng * i + r] = Wi[r] + 0.5 * dt * rate[r];
    }
}

/* ------------------------------------------------------------------------ */
/* Riemann problem in the face frame (Sec. 4)                                */
/* ------------------------------------------------------------------------ */
/* HLLC flux of the 1-D problem along x for states (rho, u, v1, v2, P), with
 * Davis wave-speed estimates and the contact speed from the Rankine-Hugoniot
 * conditions across the two outer waves. */
void orc_hllc_1d(const double *L, const double *R, double gamma, double *F)
{
    double rl = L[0], ul = L[1], pl = L[4];
    double rr = R[0], ur = R[1], pr = R[4];
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double El = pl / (gamma - 1.0) + 0.5 * rl * (ul * ul + L[2] * L[2] + L[3] * L[3]);
    double Er = pr / (gamma - 1.0) + 0.5 * rr * (ur * ur + R[2] * R[2] + R[3] * R[3]);
    double sl = fmin(ul - cl, ur - cr);
    double sr = fmax(ul + cl, ur + cr);
    double ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur));
    double Fl[5] = {rl * ul, rl * ul * ul + pl, rl * ul * L[2], rl * ul * L[3], (El + pl) * ul};
    double Fr[5] = {rr * ur, rr * ur * ur + pr, rr * ur * R[2], rr * ur * R[3], (Er + pr) * ur};
    if (sl >= 0.0) {
        memcpy(F, Fl, sizeof(Fl));
        return;
    }
    if (ss >= 0.0) {
        double Ul[5] = {rl, rl * ul, rl * L[2], rl * L[3], El};
        double f = rl * (sl - ul) / (sl - ss);
        double Us[5] = {f, f * ss, f * L[2], f * L[3], f * (El / rl + (ss - ul) * (ss + pl / (rl * (sl - ul))))};
        for (int k = 0; k < 5; ++k) F[k] = Fl[k] + sl * (Us[k] - Ul[k]);
        return;
    }
    if (sr > 0.0) {
        double Ur[5] = {rr, rr * ur, rr * R[2], rr * R[3], Er};
        double f = rr * (sr - ur) / (sr - ss);
        double Us[5] = {f, f * ss, f * R[2], f * R[3], f * (Er / rr + (ss - ur) * (ss + pr / (rr * (sr - ur))))};
        for (int k = 0; k < 5; ++k) F[k] = Fr[k] + sr * (Us[k] - Ur[k]);
        return;
    }
    memcpy(F, Fr, sizeof(Fr));
}

/* HLL flux of the same 1-D problem: the single intermediate state between
 * the Davis wave speeds, from the integral form of the conservation laws. */
void orc_hll_1d(const double *L, const double *R, double gamma, double *F)
{
    double rl = L[0], ul = L[1], pl = L[4];
    double rr = R[0], ur = R[1], pr = R[4];
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double El = pl / (gamma - 1.0) + 0.5 * rl * (ul * ul + L[2] * L[2] + L[3] * L[3]);
    double Er = pr / (gamma - 1.0) + 0.5 * rr * (ur * ur + R[2] * R[2] + R[3] * R[3]);
    double sl = fmin(ul - cl, ur - cr);
    double sr = fmax(ul + cl, ur + cr);
    double Fl[5] = {rl * ul, rl * ul * ul + pl, rl * ul * L[2], rl * ul * L[3], (El + pl) * ul};
    double Fr[5] = {rr * ur, rr * ur * ur + pr, rr * ur * R[2], rr * ur * R[3], (Er + pr) * ur};
    if (sl >= 0.0) { memcpy(F, Fl, sizeof(Fl)); return; }
    if (sr <= 0.0) { memcpy(F, Fr, sizeof(Fr)); return; }
    double Ul[5] = {rl, rl * ul, rl * L[2], rl * L[3], El};
    double Ur[5] = {rr, rr * ur, rr * R[2], rr * R[3], Er};
    for (int k = 0; k < 5; ++k) F[k] = (sr * Fl[k] - sl * Fr[k] + sl * sr * (Ur[k] - Ul[k])) / (sr - sl);
}

/* Orthonormal basis (n, t1, t2) with t1 perpendicular to n. */
static void face_basis(const double *n, double *t1, double *t2)
{
    double ax[3] = {0, 0, 0};
    if (fabs(n[0]) <= fabs(n[1]) && fabs(n[0]) <= fabs(n[2])) ax[0] = 1;
    else if (fabs(n[1]) <= fabs(n[2])) ax[1] = 1;
    else ax[2] = 1;
    cross3(n, ax, t1);
    double l = sqrt(dot3(t1, t1));
    for (int d = 0; d < 3; ++d) t1[d] /= l;
    cross3(n, t1, t2);
}

/* Contact speed S* and star pressure P* of the HLLC model: Davis wave speeds,
 * S* from the jump conditions across the outer waves, and P* from the left
 * wave's jump condition (the right one gives the same value). */
void orc_star_state(const double *L, const double *R, double gamma, double *sl, double *ss, double *sr,
                    double *pstar)
{
    double rl = L[0], ul = L[1], pl = L[4];
    double rr = R[0], ur = R[1], pr = R[4];
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    *sl = fmin(ul - cl, ur - cr);
    *sr = fmax(ul + cl, ur + cr);
    *ss = (pr - pl + rl * ul * (*sl - ul) - rr * ur * (*sr - ur)) / (rl * (*sl - ul) - rr * (*sr - ur));
    *pstar = pl + rl * (*sl - ul) * (*ss - ul);
}

/* Mach number of a shock that raises the pressure of the gas it runs into
 * from P to P_star (Rankine-Hugoniot): M^2 = 1 + (gamma+1)/(2 gamma) (P_star / P - 1).
 * The face's value is the larger over the two sides, 0 if neither is
 * compressed (Sec. 4.3 reading). */
double orc_shock_mach(const double *L, const double *R, double gamma)
{
    double sl, ss, sr, ps;
    orc_star_state(L, R, gamma, &sl, &ss, &sr, &ps);
    double m = 0.0;
    const double *side[2] = {L, R};
    for (int s = 0; s < 2; ++s) {
        double p = side[s][4];
        if (ps > p) {
            double mk = sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (ps / p - 1.0));
            if (mk > m) m = mk;
        }
    }
    return m;
}

/* Boost both per-volume states into the frame of a face moving at wface,
 * rotate so that x lies along the normal (i -> j), solve, rotate back and
 * boost the flux back into the lab frame.  With the entropy column, rho A is
 * a passive scalar: its flux is A of the upwind side times the mass flux
 * (HLLC: the side of the contact; HLL: the HLL average of rho A), and it is
 * unchanged by the boost; the face's shock Mach number goes to *mach. */
void orc_riemann_lab(const double *WL, const double *WR, const double *nrm, const double *wf,
                     const orc_cfg *cfg, double *F, double *mach)
{
    double g = cfg->gamma;
    double t1[3], t2[3];
    face_basis(nrm, t1, t2);
    double pl[5], pr[5];
    const double *Ws[2] = {WL, WR};
    double *ps[2] = {pl, pr};
    for (int s = 0; s < 2; ++s) {
        const double *W = Ws[s];
        double rho = W[0];
        double v[3] = {W[1] / rho - wf[0], W[2] / rho - wf[1], W[3] / rho - wf[2]};
        double vl[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
        double P = (g - 1.0) * (W[4] - 0.5 * rho * dot3(vl, vl));
        ps[s][0] = rho;
        ps[s][1] = dot3(v, nrm);
        ps[s][2] = dot3(v, t1);
        ps[s][3] = dot3(v, t2);
        ps[s][4] = P;
    }
    double Fp[5];
    if (cfg->riemann == 1) orc_hll_1d(pl, pr, g, Fp);
    else orc_hllc_1d(pl, pr, g, Fp);
    double fm = Fp[0];
    double fp[3];
    for (int d = 0; d < 3; ++d) fp[d] = Fp[1] * nrm[d] + Fp[2] * t1[d] + Fp[3] * t2[d];
    F[0] = fm;
    for (int d = 0; d < 3; ++d) F[1 + d] = fp[d] + fm * wf[d];
    F[4] = Fp[4] + dot3(fp, wf) + 0.5 * dot3(wf, wf) * fm;
    if (cfg->entropy) {
        double al = WL[5] / WL[0], ar = WR[5] / WR[0];
        double sl, ss, sr, pst;
        orc_star_state(pl, pr, g, &sl, &ss, &sr, &pst);
        if (cfg->riemann == 1) {
            double fl = pl[0] * pl[1] * al, fr = pr[0] * pr[1] * ar;
            if (sl >= 0.0) F[5] = fl;
            else if (sr <= 0.0) F[5] = fr;
            else F[5] = (sr * fl - sl * fr + sl * sr * (WR[5] - WL[5])) / (sr - sl);
        } else {
            F[5] = fm * ((sl >= 0.0 || ss >= 0.0) ? al : ar);
        }
    }
    if (mach) *mach = orc_shock_mach(pl, pr, g);
}

/* Face velocity (Sec. 4): mean of the two generator velocities plus the
 * correction for the face centroid lying off the generators' midpoint. */
static void face_velocity(const double *ri, const double *rj, const double *wi, const double *wj,
                          const double *fc, double *wf)
{
    double dr[3], mid[3], dw[3];
    for (int d = 0; d < 3; ++d) {
        dr[d] = rj[d] - ri[d];
        mid[d] = fc[d] - 0.5 * (ri[d] + rj[d]);
        dw[d] = wi[d] - wj[d];
    }
    double l = sqrt(dot3(dr, dr));
    double s = dot3(dw, mid) / l;
    for (int d = 0; d < 3; ++d) wf[d] = s * dr[d] / l + 0.5 * (wi[d] + wj[d]);
}

void orc_face_flux(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const int32_t *fshift,
                   const double *farea, const double *fnormal, const double *fcentroid,
                   const double *pos, const double *centroid, const double *box,
                   const double *Wh, const double *grad, const double *w, const orc_cfg *cfg,
                   double *flux, double *mach, double *vrate)
{
    (void)n;
    const int ng = state_width(cfg);
    for (int64_t f = 0; f < nf; ++f) {
        int32_t i = fi[f], j = fj[f];
        const int32_t *sh = fshift + 3 * f;
        const double *fc = fcentroid + 3 * f;
        double ci[3], cj[3], rj[3];
        for (int d = 0; d < 3; ++d) {
            ci[d] = centroid[3 * i + d];
            cj[d] = centroid[3 * j + d] + sh[d] * box[d];
            rj[d] = pos[3 * j + d] + sh[d] * box[d];
        }
        double WL[6], WR[6], WLf[6], WRf[6];
        for (int k = 0; k < ng; ++k) {
            WL[k] = Wh[ng * i + k];
            WR[k] = Wh[ng * j + k];
            for (int d = 0; d < 3; ++d) {
                WL[k] += (fc[d] - ci[d]) * grad[3 * ng * i + 3 * k + d];
                WR[k] += (fc[d] - cj[d]) * grad[3 * ng * j + 3 * k + d];
            }
        }
        orc_floor_state(WL, cfg, WLf, 0);
        orc_floor_state(WR, cfg, WRf, 0);
        if (ng == 6) {
            /* rho A at the face: a state reset to the density floor takes the
             * floor state's own A; otherwise the reconstruction, not below 0 */
            double *in[2] = {WL, WR}, *out[2] = {WLf, WRf};
            for (int s2 = 0; s2 < 2; ++s2) {
                if (!(in[s2][0] >= cfg->rho_floor)) {
                    double rf = cfg->rho_floor;
                    out[s2][5] = rf * (cfg->gamma - 1.0) * rf * cfg->eps_floor / pow(rf, cfg->gamma);
                } else {
                    out[s2][5] = in[s2][5] > 0.0 ? in[s2][5] : 0.0;
                }
            }
        }
        double wf[3];
        face_velocity(pos + 3 * i, rj, w + 3 * i, w + 3 * j, fc, wf);
        double F[6], m = 0.0;
        orc_riemann_lab(WLf, WRf, fnormal + 3 * f, wf, cfg, F, &m);
        for (int k = 0; k < ng; ++k) flux[ng * f + k] = farea[f] * F[k];
        if (mach) mach[f] = m;
        /* rate at which the moving face sweeps volume out of cell i */
        if (vrate) vrate[f] = farea[f] * dot3(wf, fnormal + 3 * f);
    }
}

/* U_i <- U_i - dt sum_{faces of i} (+/-) A F: the face flux is along the
 * normal from i to j, so it leaves i and enters j.  Then the cell floors.
 *
 * With the entropy column (Sec. 4.3), a cell whose largest face shock Mach
 * number is below mach_th takes its internal energy from the entropy,
 * E = |p|^2/(2m) + A rho^gamma V' / (gamma - 1); elsewhere the energy is kept
 * and the entropy reset from it, as is any state the floors change.  Both
 * conversions need the cell's density at the end of the step: V' = V + dt
 * sum_f (+/-) A_f (w_f . n_f) is the volume the moving faces sweep the cell
 * to (the cell's true new volume is known only after the next
 * tessellation). */
void orc_update(int64_t n, int64_t nf, const int32_t *fi, const int32_t *fj, const double *flux,
                const double *mach, const double *vrate, double dt, const double *volume, const orc_cfg *cfg,
                double *U)
{
    const int ng = state_width(cfg);
    const double g = cfg->gamma;
    double *acc = (double *)calloc(ng * n, sizeof(double));
    double *mc = (double *)calloc(n, sizeof(double));
    double *dv = (double *)calloc(n, sizeof(double));
    for (int64_t f = 0; f < nf; ++f) {
        for (int k = 0; k < ng; ++k) {
            acc[ng * fi[f] + k] += flux[ng * f + k];
            acc[ng * fj[f] + k] -= flux[ng * f + k];
        }
        if (ng == 6) {
            if (mach[f] > mc[fi[f]]) mc[fi[f]] = mach[f];
            if (mach[f] > mc[fj[f]]) mc[fj[f]] = mach[f];
            dv[fi[f]] += vrate[f];
            dv[fj[f]] -= vrate[f];
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double *u = U + ng * i;
        const double V = volume[i];
        for (int k = 0; k < ng; ++k) u[k] -= dt * acc[ng * i + k];
        int energy = 1;
        const double Vn = V + dt * dv[i];
        if (ng == 6) {
            energy = mc[i] >= cfg->mach_th;
            if (!energy) {
                if (u[0] > 0.0 && u[5] > 0.0 && Vn > 0.0) {
                    double rho = u[0] / Vn;
                    double P = (u[5] / u[0]) * pow(rho, g);
                    u[4] = 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0] + P * Vn / (g - 1.0);
                } else {
                    energy = 1;
                }
            }
        }
        double W[5], Wf[5];
        int ch = 0;
        for (int k = 0; k < 5; ++k) W[k] = u[k] / V;
        orc_floor_state(W, cfg, Wf, &ch);
        if (ch)
            for (int k = 0; k < 5; ++k) u[k] = Wf[k] * V;
        if (ng == 6 && (energy || ch)) {
            double Vr = Vn > 0.0 ? Vn : V;
            double rho = u[0] / Vr;
            double P = (g - 1.0) * (u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0]) / Vr;
            u[5] = u[0] * P / pow(rho, g);
        }
    }
    free(acc);
    free(mc);
    free(dv);
}

/* Heun's method for dU/dt = R(U, r(t)) with the generators on straight paths:
 * U* = U^n + dt R(U^n, r^n), U** = U* + dt R(U*, r^(n+1)), and
 * U^(n+1) = (U^n + U**) / 2 = U^n + dt/2 (R(U^n, r^n) + R(U*, r^(n+1))),
 * the average of the fluxes at the start and the end of the step. */
void orc_heun_average(int64_t n, const double *U0, const double *volume, const orc_cfg *cfg, double *U)
{
    for (int64_t i = 0; i < n; ++i) {
        double W[5], Wf[5];
        int ch = 0;
        for (int k = 0; k < 5; ++k) {
            U[5 * i + k] = 0.5 * (U0[5 * i + k] + U[5 * i + k]);
            W[k] = U[5 * i + k] / volume[i];
        }
        orc_floor_state(W, cfg, Wf, &ch);
        if (ch)
            for (int k = 0; k < 5; ++k) U[5 * i + k] = Wf[k] * volume[i];
    }
}

/* ------------------------------------------------------------------------ */
/* Mesh velocity, timestep, drift (Sec. 4.2)                                 */
/* ------------------------------------------------------------------------ */
static double sound_speed(const double *U, double V, double gamma)
{
    double rho = U[0] / V;
    double m2 = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / (V * V);
    double P = (gamma - 1.0) * (U[4] / V - 0.5 * m2 / rho);
    if (P < 0.0) P = 0.0;
    return sqrt(gamma * P / rho);
}

static double eff_radius(double V) { return cbrt(3.0 * V / (4.0 * M_PI)); }

void orc_mesh_velocity(int64_t n, const double *pos, const double *U, const double *volume,
                       const double *centroid, const orc_cfg *cfg, double *w)
{
    const int ng = state_width(cfg);
    for (int64_t i = 0; i < n; ++i) {
        const double *u = U + ng * i;
        for (int d = 0; d < 3; ++d) w[3 * i + d] = cfg->eta * u[1 + d] / u[0];
        if (!cfg->regularize) continue;
        double dv[3];
        for (int d = 0; d < 3; ++d) dv[d] = centroid[3 * i + d] - pos[3 * i + d];
        double dist = sqrt(dot3(dv, dv));
        double R = eff_radius(volume[i]);
        double zr = cfg->zeta * R;
        double ramp;
        if (dist < 0.9 * zr) ramp = 0.0;
        else if (dist > 1.1 * zr) ramp = 1.0;
        else ramp = (dist - 0.9 * zr) / (0.2 * zr);
        if (ramp > 0.0 && dist > 0.0) {
            double cs = sound_speed(u, volume[i], cfg->gamma);
            for (int d = 0; d < 3; ++d) w[3 * i + d] += cfg->chi * cs * ramp * dv[d] / dist;
        }
    }
}

double orc_timestep(int64_t n, const double *U, const double *volume, const double *w,
                    const orc_cfg *cfg)
{
    const int ng = state_width(cfg);
    double dt = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        const double *u = U + ng * i;
        double cs = sound_speed(u, volume[i], cfg->gamma);
        double rel[3];
        for (int d = 0; d < 3; ++d) rel[d] = u[1 + d] / u[0] - w[3 * i + d];
        double t = cfg->cfl * eff_radius(volume[i]) / (cs + sqrt(dot3(rel, rel)));
        if (t < dt) dt = t;
    }
    return dt;
}

void orc_drift(int64_t n, double *pos, const double *w, double dt, const double *box)
{
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            double x = fmod(pos[3 * i + d] + w[3 * i + d] * dt, box[d]);
            if (x < 0.0) x += box[d];
            if (x >= box[d]) x -= box[d];
            pos[3 * i + d] = x;
        }
}
