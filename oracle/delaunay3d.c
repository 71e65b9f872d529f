/*
 * delaunay3d.c -- the oracle's own 3-D Delaunay tetrahedralisation.
 * TEST INFRASTRUCTURE ONLY (cross-checks the QHull grids the inputs use).
 *
 * Sect. 2.1.2: the Delaunay triangulation of the grid points is the set of
 * tetrahedra whose circumspheres contain no other point (empty circumsphere
 * criterion).  This is incremental Bowyer-Watson insertion: find the
 * tetrahedra whose circumsphere contains the new point (the cavity), delete
 * them and connect the point to the cavity boundary.  The convex hull is
 * handled with one symbolic vertex at infinity: a tetrahedron (a,b,c,INF)
 * stands for the outside of hull facet (a,b,c) and is in conflict with every
 * point strictly beyond that facet.  Plain double predicates: fine for points
 * in general position (random inputs), not for degenerate sets.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define INF_V (-1)

typedef struct {
    int32_t v[4];
    int32_t nb[4]; /* nb[j] shares the face opposite v[j] */
    int alive;
} tet_t;

typedef struct {
    const double *p;
    tet_t *t;
    int64_t nt, cap;
} mesh_t;

/* orient(a,b,c,d) = ((b-a) x (c-a)) . (d-a) */
static double orient(const double *a, const double *b, const double *c, const double *d) {
    double bx = b[0] - a[0], by = b[1] - a[1], bz = b[2] - a[2];
    double cx = c[0] - a[0], cy = c[1] - a[1], cz = c[2] - a[2];
    double dx = d[0] - a[0], dy = d[1] - a[1], dz = d[2] - a[2];
    return (by * cz - bz * cy) * dx + (bz * cx - bx * cz) * dy + (bx * cy - by * cx) * dz;
}

/* > 0 iff e lies inside the circumsphere of (a,b,c,d), any orientation. */
static double insphere_signed(const double *a, const double *b, const double *c, const double *d,
                              const double *e) {
    double m[4][4];
    const double *pts[4] = {a, b, c, d};
    for (int i = 0; i < 4; ++i) {
        double x = pts[i][0] - e[0], y = pts[i][1] - e[1], z = pts[i][2] - e[2];
        m[i][0] = x; m[i][1] = y; m[i][2] = z; m[i][3] = x * x + y * y + z * z;
    }
    /* 4x4 determinant by cofactor expansion along column 3 */
    double det = 0.0;
    for (int i = 0; i < 4; ++i) {
        double s[3][3];
        int r = 0;
        for (int k = 0; k < 4; ++k) {
            if (k == i) continue;
            s[r][0] = m[k][0]; s[r][1] = m[k][1]; s[r][2] = m[k][2];
            r++;
        }
        double minor = s[0][0] * (s[1][1] * s[2][2] - s[1][2] * s[2][1]) -
                       s[0][1] * (s[1][0] * s[2][2] - s[1][2] * s[2][0]) +
                       s[0][2] * (s[1][0] * s[2][1] - s[1][1] * s[2][0]);
        double sign = ((i + 3) % 2 == 0) ? 1.0 : -1.0;
        det += sign * m[i][3] * minor;
    }
    /* det > 0 means inside when orient(a,b,c,d) < 0 in the convention above */
    double o = orient(a, b, c, d);
    return -det * (o > 0 ? 1.0 : -1.0);
}

static const double *P(const mesh_t *m, int32_t v) { return m->p + 3 * (int64_t)v; }

static int has_inf(const tet_t *t) {
    return t->v[0] == INF_V || t->v[1] == INF_V || t->v[2] == INF_V || t->v[3] == INF_V;
}

/* orientation of tet t with vertex slot j replaced by point q (INF must not remain) */
static double orient_replace(const mesh_t *m, const tet_t *t, int j, const double *q) {
    const double *pp[4];
    for (int i = 0; i < 4; ++i) pp[i] = (i == j) ? q : P(m, t->v[i]);
    return orient(pp[0], pp[1], pp[2], pp[3]);
}

static int conflict(const mesh_t *m, const tet_t *t, const double *q) {
    for (int j = 0; j < 4; ++j)
        if (t->v[j] == INF_V) return orient_replace(m, t, j, q) > 0.0;
    return insphere_signed(P(m, t->v[0]), P(m, t->v[1]), P(m, t->v[2]), P(m, t->v[3]), q) > 0.0;
}

static int64_t new_tet(mesh_t *m) {
    if (m->nt == m->cap) {
        m->cap = m->cap ? 2 * m->cap : 1024;
        m->t = (tet_t *)realloc(m->t, sizeof(tet_t) * (size_t)m->cap);
    }
    int64_t id = m->nt++;
    m->t[id].alive = 1;
    for (int j = 0; j < 4; ++j) m->t[id].nb[j] = -1;
    return id;
}

static int slot_of(const tet_t *t, int32_t v) {
    for (int j = 0; j < 4; ++j)
        if (t->v[j] == v) return j;
    return -1;
}

/* walk towards q; return a tetrahedron in conflict with q (or -1) */
static int64_t locate(const mesh_t *m, int64_t start, const double *q) {
    int64_t cur = start;
    for (int64_t steps = 0; steps < 4 * m->nt + 16; ++steps) {
        const tet_t *t = &m->t[cur];
        if (has_inf(t)) {
            if (conflict(m, t, q)) return cur;
            int j = slot_of(t, INF_V);
            cur = t->nb[j];
            continue;
        }
        int moved = 0;
        for (int j = 0; j < 4; ++j) {
            if (orient_replace(m, t, j, q) < 0.0) {
                cur = t->nb[j];
                moved = 1;
                break;
            }
        }
        if (!moved) return cur;
    }
    return -1;
}

/*
 * Triangulate n points (xyz, row-major).  On success returns the number of
 * finite tetrahedra written to *tets_out (malloc'ed int32 [ntet*4], caller
 * frees with dl_free); returns -1 if the first points are degenerate.
 */
int64_t dl_triangulate(int64_t n, const double *pts, int32_t **tets_out) {
    mesh_t m = {pts, NULL, 0, 0};
    *tets_out = NULL;
    if (n < 4) return -1;
    /* initial tetrahedron: points 0,1,2 and the first non-coplanar one */
    int64_t i3 = -1;
    for (int64_t i = 3; i < n; ++i)
        if (orient(P(&m, 0), P(&m, 1), P(&m, 2), P(&m, (int32_t)i)) != 0.0) {
            i3 = i;
            break;
        }
    if (i3 < 0) return -1;
    int32_t a = 0, b = 1, c = 2, d = (int32_t)i3;
    if (orient(P(&m, a), P(&m, b), P(&m, c), P(&m, d)) < 0.0) {
        int32_t tmp = a; a = b; b = tmp;
    }
    int64_t t0 = new_tet(&m);
    m.t[t0].v[0] = a; m.t[t0].v[1] = b; m.t[t0].v[2] = c; m.t[t0].v[3] = d;
    /* one infinite tet per face; replacing INF by a point beyond the face
       gives positive orientation, matching the finite tet with that slot
       replaced by the point */
    for (int j = 0; j < 4; ++j) {
        int64_t ti = new_tet(&m);
        tet_t *T = &m.t[ti];
        memcpy(T->v, m.t[t0].v, sizeof(T->v));
        /* face opposite j seen from outside: swap two other vertices, INF at slot j */
        T->v[j] = INF_V;
        int o1 = (j + 1) % 4, o2 = (j + 2) % 4;
        int32_t tmp = T->v[o1]; T->v[o1] = T->v[o2]; T->v[o2] = tmp;
        T->nb[j] = (int32_t)t0;
        m.t[t0].nb[j] = (int32_t)ti;
    }
    /* link infinite tets with each other across faces containing INF */
    for (int64_t x = 1; x <= 4; ++x)
        for (int jx = 0; jx < 4; ++jx) {
            if (m.t[x].v[jx] == INF_V) continue;
            /* face of x opposite jx contains INF; find the other infinite tet with that face */
            int32_t fv[3];
            int r = 0;
            for (int k = 0; k < 4; ++k)
                if (k != jx) fv[r++] = m.t[x].v[k];
            for (int64_t y = 1; y <= 4; ++y) {
                if (y == x) continue;
                int cnt = 0;
                for (int k = 0; k < 3; ++k) cnt += slot_of(&m.t[y], fv[k]) >= 0;
                if (cnt == 3) {
                    m.t[x].nb[jx] = (int32_t)y;
                    break;
                }
            }
        }

    int64_t last = t0;
    int64_t *stack = NULL, *cav = NULL;
    int64_t scap = 0, ccap = 0;
    char *mark = NULL;
    int64_t mcap = 0;
    for (int64_t ip = 0; ip < n; ++ip) {
        if (ip == a || ip == b || ip == c || ip == d) continue;
        const double *q = P(&m, (int32_t)ip);
        int64_t seed = locate(&m, last, q);
        if (seed < 0 || !conflict(&m, &m.t[seed], q)) {
            seed = -1;
            for (int64_t k = 0; k < m.nt; ++k)
                if (m.t[k].alive && conflict(&m, &m.t[k], q)) {
                    seed = k;
                    break;
                }
            if (seed < 0) continue; /* duplicate point */
        }
        if (mcap < m.nt + 64) {
            int64_t nc = 2 * (m.nt + 64);
            mark = (char *)realloc(mark, (size_t)nc);
            memset(mark + mcap, 0, (size_t)(nc - mcap));
            mcap = nc;
        }
        /* cavity by flood fill over conflicting neighbours */
        int64_t ns = 0, nc = 0;
        if (scap < 64) { scap = 64; stack = (int64_t *)realloc(stack, sizeof(int64_t) * scap); }
        stack[ns++] = seed;
        mark[seed] = 1;
        while (ns) {
            int64_t cur = stack[--ns];
            if (nc == ccap) { ccap = ccap ? 2 * ccap : 64; cav = (int64_t *)realloc(cav, sizeof(int64_t) * ccap); }
            cav[nc++] = cur;
            for (int j = 0; j < 4; ++j) {
                int64_t nbt = m.t[cur].nb[j];
                if (nbt < 0 || mark[nbt]) continue;
                if (conflict(&m, &m.t[nbt], q)) {
                    mark[nbt] = 1;
                    if (ns == scap) { scap *= 2; stack = (int64_t *)realloc(stack, sizeof(int64_t) * scap); }
                    stack[ns++] = nbt;
                }
            }
        }
        /* new tets on the cavity boundary */
        int64_t first_new = m.nt;
        for (int64_t ci = 0; ci < nc; ++ci) {
            int64_t cur = cav[ci];
            for (int j = 0; j < 4; ++j) {
                int64_t nbt = m.t[cur].nb[j];
                if (nbt >= 0 && mark[nbt] == 1) continue; /* interior face */
                int64_t nt_id = new_tet(&m);
                if (mcap < m.nt + 64) {
                    int64_t ncap = 2 * (m.nt + 64);
                    mark = (char *)realloc(mark, (size_t)ncap);
                    memset(mark + mcap, 0, (size_t)(ncap - mcap));
                    mcap = ncap;
                }
                tet_t *T = &m.t[nt_id];
                memcpy(T->v, m.t[cur].v, sizeof(T->v));
                T->v[j] = (int32_t)ip;
                T->nb[j] = (int32_t)nbt;
                if (nbt >= 0) {
                    /* back-link: the face of nbt shared with cur */
                    for (int k = 0; k < 4; ++k)
                        if (m.t[nbt].nb[k] == cur) m.t[nbt].nb[k] = (int32_t)nt_id;
                }
            }
        }
        /* link new tets to each other: faces containing ip */
        for (int64_t x = first_new; x < m.nt; ++x) {
            int jp = slot_of(&m.t[x], (int32_t)ip);
            for (int jx = 0; jx < 4; ++jx) {
                if (jx == jp) continue;                   /* the cavity-boundary face */
                if (m.t[x].nb[jx] >= first_new) continue; /* already linked from its partner */
                int32_t fv[2];
                int r = 0;
                for (int k = 0; k < 4; ++k)
                    if (k != jx && k != jp) fv[r++] = m.t[x].v[k];
                for (int64_t y = first_new; y < m.nt; ++y) {
                    if (y == x) continue;
                    if (slot_of(&m.t[y], fv[0]) >= 0 && slot_of(&m.t[y], fv[1]) >= 0) {
                        int jy = -1;
                        for (int k = 0; k < 4; ++k) {
                            int32_t vv = m.t[y].v[k];
                            if (vv != fv[0] && vv != fv[1] && vv != (int32_t)ip) jy = k;
                        }
                        m.t[x].nb[jx] = (int32_t)y;
                        m.t[y].nb[jy] = (int32_t)x;
                        break;
                    }
                }
            }
        }
        for (int64_t ci = 0; ci < nc; ++ci) {
            m.t[cav[ci]].alive = 0;
            mark[cav[ci]] = 2; /* dead: never revisited */
        }
        last = m.nt - 1;
    }
    free(stack); free(cav); free(mark);
    int64_t nfin = 0;
    for (int64_t k = 0; k < m.nt; ++k)
        if (m.t[k].alive && !has_inf(&m.t[k])) nfin++;
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(nfin ? nfin : 1));
    int64_t w = 0;
    for (int64_t k = 0; k < m.nt; ++k)
        if (m.t[k].alive && !has_inf(&m.t[k])) {
            memcpy(out + 4 * w, m.t[k].v, sizeof(int32_t) * 4);
            w++;
        }
    free(m.t);
    *tets_out = out;
    return nfin;
}

void dl_free(int32_t *p) { free(p); }

/* 1 if e is strictly inside the circumsphere of (a,b,c,d). */
int dl_insphere(const double *a, const double *b, const double *c, const double *d,
                const double *e) {
    return insphere_signed(a, b, c, d, e) > 0.0;
}
