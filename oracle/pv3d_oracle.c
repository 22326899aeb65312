/*
 * pv3d_oracle.c -- FP64 CPU oracle for the 3DPV shadow-sample path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes (Robledo, Leloux & Lorenzo, "3D simulation of complex
 * shading affecting PV systems ...", Section 2):
 *   Step 2   PV generator: modules with an n_u x n_v cell grid, a bypass
 *            substring per cell, fixed or carried by a two-axis tracker.
 *   Step 3   Shading: the paper approximates, by shadow mapping, the plain
 *            definition "a point of the generator is shaded iff the ray from it
 *            toward the sun meets an object of the scene".  The oracle evaluates
 *            that definition exactly: a Moller-Trumbore (1997) ray/triangle test
 *            in FP64 for every sub-cell sample, accelerated by a median-split
 *            bounding-volume hierarchy (brute force is selectable).
 *   Step 3   Sub-cell areas: n x n samples per cell at cell-local ((i+1/2)/n,
 *            (j+1/2)/n) -- the cell centre for n = 1, the 3x3 areas for n = 3.
 *   Step 4   Geometric shading removes the beam component from shaded areas;
 *            the effective (electrical) shading uses a series-current-limited
 *            bypass-diode model (the paper cites a diode model and a system model
 *            without giving them) and per-step losses are integrated over time.
 *
 * Besides the flags the oracle can mark samples whose shadow-map answer is
 * ambiguous at one texel of resolution (the parity mask): a sample is masked if
 * the light-space projection of the part of some other triangle lying in front
 * of the sample's own module plane has an edge within one texel of the sample,
 * or covers it at a depth gap smaller than the texel-scale depth swing.
 * Texel size and the light frame follow the orthographic sun view whose field
 * of view is limited to the generator (Section 2, step 3).
 *
 * parity pins: brute force vs BVH; closed-form pole, convex-obstacle and
 * infinite-sheds shadows; PV-model closed forms; the per-cell beam loss under
 * a straight shadow edge; tracker cell centres about the pivot at right-angle
 * poses; invariants (tests/).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------------- */
/* small FP64 vector algebra                                                  */
/* ------------------------------------------------------------------------- */
typedef struct { double x, y, z; } vec3;

static vec3 mk(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 add(vec3 a, vec3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 sub(vec3 a, vec3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 scl(vec3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 cross(vec3 a, vec3 b)
{
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(vec3 a) { return sqrt(dot(a, a)); }
static vec3 unit(vec3 a) { return scl(a, 1.0 / len(a)); }
static double comp(vec3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

typedef struct { vec3 p[3]; } tri_t;

/* ------------------------------------------------------------------------- */
/* bounding-volume hierarchy, median split on the longest centroid axis       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double lo[3], hi[3];
    int32_t left;   /* inner node: index of the first child (second = left + 1) */
    int32_t first;  /* leaf: first entry of `order` */
    int32_t count;  /* leaf: number of triangles (0 = inner node) */
} node_t;

typedef struct {
    const tri_t* tris;
    int32_t n_tris;
    int32_t* order;
    node_t* nodes;
    int32_t n_nodes, cap_nodes;
    double* cen;  /* centroids, 3 per triangle */
} bvh_t;

static void tri_bounds(const tri_t* t, double lo[3], double hi[3])
{
    for (int k = 0; k < 3; ++k) {
        double a = comp(t->p[0], k), b = comp(t->p[1], k), c = comp(t->p[2], k);
        lo[k] = fmin(a, fmin(b, c));
        hi[k] = fmax(a, fmax(b, c));
    }
}

static void swap_i(int32_t* a, int32_t* b) { int32_t t = *a; *a = *b; *b = t; }

/* Reorder order[lo..hi) so that position `k` holds its sorted element along `axis`. */
static void select_kth(bvh_t* b, int32_t lo, int32_t hi, int32_t k, int axis)
{
    while (hi - lo > 1) {
        int32_t mid = lo + (hi - lo) / 2;
        double pivot = b->cen[3 * b->order[mid] + axis];
        int32_t i = lo, j = hi - 1;
        while (i <= j) {
            while (b->cen[3 * b->order[i] + axis] < pivot) ++i;
            while (b->cen[3 * b->order[j] + axis] > pivot) --j;
            if (i <= j) { swap_i(&b->order[i], &b->order[j]); ++i; --j; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static int32_t bvh_new_node(bvh_t* b)
{
    if (b->n_nodes == b->cap_nodes) {
        b->cap_nodes = b->cap_nodes ? 2 * b->cap_nodes : 64;
        b->nodes = (node_t*)realloc(b->nodes, sizeof(node_t) * (size_t)b->cap_nodes);
    }
    return b->n_nodes++;
}

static void bvh_build_rec(bvh_t* b, int32_t ni, int32_t lo, int32_t hi)
{
    node_t* nd = &b->nodes[ni];
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < 3; ++k) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    for (int32_t i = lo; i < hi; ++i) {
        double tlo[3], thi[3];
        tri_bounds(&b->tris[b->order[i]], tlo, thi);
        for (int k = 0; k < 3; ++k) {
            nd->lo[k] = fmin(nd->lo[k], tlo[k]);
            nd->hi[k] = fmax(nd->hi[k], thi[k]);
            double c = b->cen[3 * b->order[i] + k];
            clo[k] = fmin(clo[k], c);
            chi[k] = fmax(chi[k], c);
        }
    }
    int32_t n = hi - lo;
    int axis = 0;
    double ext = chi[0] - clo[0];
    if (chi[1] - clo[1] > ext) { axis = 1; ext = chi[1] - clo[1]; }
    if (chi[2] - clo[2] > ext) { axis = 2; ext = chi[2] - clo[2]; }
    if (n <= 4 || ext <= 0.0) {
        nd->count = n; nd->first = lo; nd->left = -1;
        return;
    }
    int32_t mid = lo + n / 2;
    select_kth(b, lo, hi, mid, axis);
    int32_t l = bvh_new_node(b);
    int32_t r = bvh_new_node(b);
    (void)r;
    b->nodes[ni].count = 0;
    b->nodes[ni].left = l;
    b->nodes[ni].first = -1;
    bvh_build_rec(b, l, lo, mid);
    bvh_build_rec(b, l + 1, mid, hi);
}

static void bvh_build(bvh_t* b, const tri_t* tris, int32_t n)
{
    memset(b, 0, sizeof(*b));
    b->tris = tris;
    b->n_tris = n;
    if (n == 0) return;
    b->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    b->cen = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        b->order[i] = i;
        vec3 c = scl(add(add(tris[i].p[0], tris[i].p[1]), tris[i].p[2]), 1.0 / 3.0);
        b->cen[3 * i] = c.x; b->cen[3 * i + 1] = c.y; b->cen[3 * i + 2] = c.z;
    }
    int32_t root = bvh_new_node(b);
    bvh_build_rec(b, root, 0, n);
    free(b->cen);
    b->cen = NULL;
}

static void bvh_free(bvh_t* b)
{
    free(b->order);
    free(b->nodes);
    free(b->cen);
    memset(b, 0, sizeof(*b));
}

/* Does the segment o + t d, t in [t0, t1], pass within the box grown by r? */
static int seg_box(const node_t* nd, vec3 o, vec3 d, double r, double t0, double t1)
{
    for (int k = 0; k < 3; ++k) {
        double ok = comp(o, k), dk = comp(d, k);
        double lo = nd->lo[k] - r, hi = nd->hi[k] + r;
        if (dk == 0.0) {
            if (ok < lo || ok > hi) return 0;
            continue;
        }
        double ta = (lo - ok) / dk, tb = (hi - ok) / dk;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Moller-Trumbore ray/triangle intersection in FP64 (inclusive edges)         */
/* ------------------------------------------------------------------------- */
static int ray_hits(const tri_t* t, vec3 o, vec3 d, double t_min)
{
    vec3 e1 = sub(t->p[1], t->p[0]);
    vec3 e2 = sub(t->p[2], t->p[0]);
    vec3 pv = cross(d, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    vec3 tv = sub(o, t->p[0]);
    double a = dot(tv, pv) * inv;
    if (a < 0.0 || a > 1.0) return 0;
    vec3 qv = cross(tv, e1);
    double b = dot(d, qv) * inv;
    if (b < 0.0 || a + b > 1.0) return 0;
    double th = dot(e2, qv) * inv;
    return th > t_min;
}

/* any hit along o + t d, t > t_min, skipping triangle ids skip0 and skip1 */
static int bvh_occluded(const bvh_t* b, vec3 o, vec3 d, double t_min, int32_t skip0, int32_t skip1)
{
    if (b->n_tris == 0) return 0;
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const node_t* nd = &b->nodes[stack[--sp]];
        if (!seg_box(nd, o, d, 0.0, t_min, INFINITY)) continue;
        if (nd->count) {
            for (int32_t i = 0; i < nd->count; ++i) {
                int32_t id = b->order[nd->first + i];
                if (id == skip0 || id == skip1) continue;
                if (ray_hits(&b->tris[id], o, d, t_min)) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->left + 1;
        }
    }
    return 0;
}

static int brute_occluded(const tri_t* tris, int32_t n, vec3 o, vec3 d, double t_min,
                          int32_t skip0, int32_t skip1)
{
    for (int32_t id = 0; id < n; ++id) {
        if (id == skip0 || id == skip1) continue;
        if (ray_hits(&tris[id], o, d, t_min)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* parity mask: ambiguity of the one-texel shadow-map answer                   */
/* ------------------------------------------------------------------------- */
typedef struct {
    vec3 p, s, u, v, n;  /* sample, sun, light-plane basis, own module unit normal */
    double delta;        /* texel size */
    double g_own;        /* tan of the incidence angle on the own module */
    double eps_h;        /* thickness of the own plane */
} mask_q;

static double seg_dist2(double ax, double ay, double bx, double by)
{
    /* squared distance from the origin to segment a-b */
    double dx = bx - ax, dy = by - ay;
    double l2 = dx * dx + dy * dy;
    double t = l2 > 0.0 ? -(ax * dx + ay * dy) / l2 : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double qx = ax + t * dx, qy = ay + t * dy;
    return qx * qx + qy * qy;
}

/* 1 if triangle `t` makes sample q ambiguous at one texel */
static int mask_triangle(const tri_t* t, const mask_q* q)
{
    double a[3], b[3], h[3];
    for (int k = 0; k < 3; ++k) {
        vec3 x = sub(t->p[k], q->p);
        a[k] = dot(x, q->u);
        b[k] = dot(x, q->v);
        h[k] = dot(x, q->n);
    }
    /* clip the triangle to the side of the own plane that faces the sun */
    double pa[6], pb[6];
    int m = 0;
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3;
        int in0 = h[k] >= q->eps_h, in1 = h[k1] >= q->eps_h;
        if (in0) { pa[m] = a[k]; pb[m] = b[k]; ++m; }
        if (in0 != in1) {
            double w = (q->eps_h - h[k]) / (h[k1] - h[k]);
            pa[m] = a[k] + w * (a[k1] - a[k]);
            pb[m] = b[k] + w * (b[k1] - b[k]);
            ++m;
        }
    }
    if (m == 0) return 0;
    double d2 = q->delta * q->delta;
    if (m == 1) return pa[0] * pa[0] + pb[0] * pb[0] < d2;
    /* edge rule: an edge of the projected front part within one texel */
    for (int k = 0; k < m; ++k) {
        int k1 = (k + 1) % m;
        if (seg_dist2(pa[k], pb[k], pa[k1], pb[k1]) < d2) return 1;
    }
    if (m < 3) return 0;
    /* depth-gap rule: the front part covers the sample with a small gap */
    int pos = 0, neg = 0;
    for (int k = 0; k < m; ++k) {
        int k1 = (k + 1) % m;
        double c = pa[k] * pb[k1] - pb[k] * pa[k1];  /* origin side of edge k */
        if (c > 0) ++pos;
        if (c < 0) ++neg;
    }
    if (pos && neg) return 0;  /* origin outside the convex polygon */
    vec3 mn = cross(sub(t->p[1], t->p[0]), sub(t->p[2], t->p[0]));
    double ml = len(mn);
    if (ml == 0.0) return 0;
    mn = scl(mn, 1.0 / ml);
    double ms = dot(mn, q->s);
    if (ms == 0.0) return 0;
    double t_hit = dot(mn, sub(t->p[0], q->p)) / ms;
    double g_t = sqrt(fmax(0.0, 1.0 - ms * ms)) / fabs(ms);
    double tau = sqrt(2.0) * q->delta * (q->g_own + g_t) + q->delta / 8.0;
    return t_hit < tau;
}

static int bvh_masked(const bvh_t* b, const mask_q* q, double t_lo, int32_t skip0, int32_t skip1)
{
    if (b->n_tris == 0) return 0;
    int32_t stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const node_t* nd = &b->nodes[stack[--sp]];
        if (!seg_box(nd, q->p, q->s, q->delta, t_lo, INFINITY)) continue;
        if (nd->count) {
            for (int32_t i = 0; i < nd->count; ++i) {
                int32_t id = b->order[nd->first + i];
                if (id == skip0 || id == skip1) continue;
                if (mask_triangle(&b->tris[id], q)) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->left + 1;
        }
    }
    return 0;
}

static int brute_masked(const tri_t* tris, int32_t n, const mask_q* q, int32_t skip0, int32_t skip1)
{
    for (int32_t id = 0; id < n; ++id) {
        if (id == skip0 || id == skip1) continue;
        if (mask_triangle(&tris[id], q)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* PV electrical model (Section 2, step 4): series-current-limited cells,      */
/* one bypass diode per substring, maximum power point of the module           */
/* ------------------------------------------------------------------------- */
/*
 * Cell photocurrent I_c = i_ref * G_c / 1000.  A substring k of n_k cells in
 * series carries at most I_k = min over its cells of I_c and then delivers
 * V_k = n_k * v_cell; at a string current I above I_k its bypass diode conducts
 * and the substring costs v_diode.  P(I) = I * (sum_{k: I_k >= I} V_k
 * - v_diode * #{k: I_k < I}) is linear between consecutive I_k, so the maximum
 * power point is the best of the I_k (and 0).
 */
double pv3d_oracle_module_pmpp(int32_t n_cells, const double* g, const int32_t* cell_sub,
                               int32_t n_sub, double i_ref, double v_cell, double v_diode)
{
    double ik[64];
    int32_t nk[64];
    if (n_sub > 64) return NAN;
    for (int k = 0; k < n_sub; ++k) { ik[k] = INFINITY; nk[k] = 0; }
    for (int32_t c = 0; c < n_cells; ++c) {
        int k = cell_sub[c];
        double ic = i_ref * g[c] / 1000.0;
        if (ic < ik[k]) ik[k] = ic;
        nk[k] += 1;
    }
    double best = 0.0;
    for (int k = 0; k < n_sub; ++k) {
        if (nk[k] == 0) continue;
        double cur = ik[k];
        double volt = 0.0;
        for (int j = 0; j < n_sub; ++j) {
            if (nk[j] == 0) continue;
            if (ik[j] >= cur) volt += nk[j] * v_cell;
            else volt -= v_diode;
        }
        double p = cur * volt;
        if (p > best) best = p;
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* scene handle                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    tri_t* tris;
    int32_t n_tris;
    bvh_t bvh;
    double lo[3], hi[3];
} oscene_t;

void* pv3d_oracle_scene_create(const float* verts, int64_t n_verts, const int32_t* idx, int64_t n_tris)
{
    oscene_t* sc = (oscene_t*)calloc(1, sizeof(oscene_t));
    sc->n_tris = (int32_t)n_tris;
    sc->tris = (tri_t*)malloc(sizeof(tri_t) * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int k = 0; k < 3; ++k) { sc->lo[k] = INFINITY; sc->hi[k] = -INFINITY; }
    for (int64_t t = 0; t < n_tris; ++t) {
        for (int k = 0; k < 3; ++k) {
            int64_t vi = idx[3 * t + k];
            if (vi < 0 || vi >= n_verts) { vi = 0; }
            vec3 p = mk(verts[3 * vi], verts[3 * vi + 1], verts[3 * vi + 2]);
            sc->tris[t].p[k] = p;
            for (int a = 0; a < 3; ++a) {
                sc->lo[a] = fmin(sc->lo[a], comp(p, a));
                sc->hi[a] = fmax(sc->hi[a], comp(p, a));
            }
        }
    }
    bvh_build(&sc->bvh, sc->tris, sc->n_tris);
    return sc;
}

void pv3d_oracle_scene_destroy(void* h)
{
    oscene_t* sc = (oscene_t*)h;
    if (!sc) return;
    bvh_free(&sc->bvh);
    free(sc->tris);
    free(sc);
}

/* ------------------------------------------------------------------------- */
/* evaluation                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    /* generator */
    int32_t n_mods;
    const float* mod_f;     /* per module: origin[3], u[3], v[3], pitch */
    const int32_t* mod_i;   /* per module: cells_u, cells_v, layout, tracker, string */
    const int32_t* lay_off; /* per layout: offset into lay_sub */
    const int32_t* lay_nsub;
    const int32_t* lay_sub;
    int32_t n_trk;
    const float* pivots;    /* per tracker: xyz */
    /* sun */
    const double* sun;      /* per step: xyz */
    const float* dni, * dhi, * dt;
    const float* poses;     /* per step, per tracker: azimuth, tilt (radians) */
    /* parameters */
    int32_t n;              /* samples per cell side */
    int32_t map_res;        /* R: shadow-map side, used for the texel size */
    double i_ref, v_cell, v_diode;
    int32_t want_mask, brute;
} ogen_t;

typedef struct {
    vec3 o, u, v, n;        /* posed origin, axes, unit normal */
    vec3 c[4];              /* corners */
} posed_t;

/* Rotation of a two-axis tracker: tilt `tilt` about the east axis (the rest
 * normal +z leans toward -y), then turn about +z so the normal faces the
 * compass azimuth `az`:  R = Rz(pi - az) * Rx(tilt). */
static vec3 tracker_rotate(vec3 x, double az, double tilt)
{
    double cb = cos(tilt), sb = sin(tilt);
    vec3 y = mk(x.x, cb * x.y - sb * x.z, sb * x.y + cb * x.z);
    double g = M_PI - az;
    double cg = cos(g), sg = sin(g);
    return mk(cg * y.x - sg * y.y, sg * y.x + cg * y.y, y.z);
}

static void pose_module(const ogen_t* g, int32_t m, int64_t step, posed_t* out)
{
    const float* f = g->mod_f + 10 * (size_t)m;
    const int32_t* i = g->mod_i + 5 * (size_t)m;
    vec3 o = mk(f[0], f[1], f[2]), u = mk(f[3], f[4], f[5]), v = mk(f[6], f[7], f[8]);
    int32_t trk = i[3];
    if (trk >= 0) {
        const float* pz = g->poses + 2 * ((size_t)step * (size_t)g->n_trk + (size_t)trk);
        double az = pz[0], tilt = pz[1];
        vec3 piv = mk(g->pivots[3 * trk], g->pivots[3 * trk + 1], g->pivots[3 * trk + 2]);
        o = add(piv, tracker_rotate(o, az, tilt));
        u = tracker_rotate(u, az, tilt);
        v = tracker_rotate(v, az, tilt);
    }
    double lu = i[0] * (double)f[9], lv = i[1] * (double)f[9];
    out->o = o; out->u = u; out->v = v;
    out->n = unit(cross(u, v));
    out->c[0] = o;
    out->c[1] = add(o, scl(u, lu));
    out->c[2] = add(add(o, scl(u, lu)), scl(v, lv));
    out->c[3] = add(o, scl(v, lv));
}

/* Orthographic light frame: w = s, u = normalize(s x z) (x if the sun is at the
 * zenith), v = s x u.  Window = bounding box of the projected module corners,
 * squared to the larger side and padded by one texel on each side: texel size
 * delta = extent / (R - 2). */
static void light_frame(vec3 s, vec3* u, vec3* v)
{
    double h2 = s.x * s.x + s.y * s.y;
    *u = h2 < 1e-12 ? mk(1, 0, 0) : unit(mk(s.y, -s.x, 0.0));
    *v = cross(s, *u);
}

typedef struct {
    const oscene_t* sc;
    const ogen_t* g;
    const posed_t* posed;   /* all modules at this step */
    const tri_t* mtris;     /* module triangles at this step, 2 per module */
    const bvh_t* mbvh;
    vec3 s, lu, lv;
    double delta, t_eps, eps_h;
    const int32_t* eval_mods;
    const int64_t* cell_off;  /* per evaluated module: first cell index */
    int32_t n_eval;
    /* work queue over (evaluated module, cell row) */
    int64_t n_items;
    int64_t next;
    /* per evaluated module outputs for this step */
    int32_t* counts;        /* per evaluated cell */
    uint64_t* bits;         /* per evaluated cell (may be NULL) */
    uint64_t* mbits;        /* per evaluated cell (may be NULL) */
    const int32_t* item_mod;  /* evaluated module of each work item */
    const int32_t* item_row;  /* cell row of each work item */
} job_t;

static void eval_cell_row(job_t* J, int32_t e, int32_t cv)
{
    const ogen_t* g = J->g;
    int32_t m = J->eval_mods[e];
    const posed_t* P = &J->posed[m];
    const float* f = g->mod_f + 10 * (size_t)m;
    const int32_t* mi = g->mod_i + 5 * (size_t)m;
    int32_t cu_n = mi[0];
    double pitch = f[9];
    int n = g->n;
    double c_inc = dot(P->n, J->s);
    int maskable = J->g->want_mask && c_inc > cos(89.0 * M_PI / 180.0);
    double g_own = c_inc > 0 ? sqrt(fmax(0.0, 1.0 - c_inc * c_inc)) / c_inc : INFINITY;
    mask_q q;
    q.s = J->s; q.u = J->lu; q.v = J->lv; q.n = P->n;
    q.delta = J->delta; q.g_own = g_own; q.eps_h = J->eps_h;
    double t_lo = -J->delta * (g_own + 1.0);
    int32_t skip0 = 2 * m, skip1 = 2 * m + 1;
    for (int32_t cu = 0; cu < cu_n; ++cu) {
        int64_t cell = J->cell_off[e] + (int64_t)cv * cu_n + cu;
        int32_t cnt = 0;
        uint64_t bits = 0, mbits = 0;
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) {
                double a = (cu + (i + 0.5) / n) * pitch;
                double b = (cv + (j + 0.5) / n) * pitch;
                vec3 p = add(add(P->o, scl(P->u, a)), scl(P->v, b));
                int hit;
                if (g->brute)
                    hit = brute_occluded(J->sc->tris, J->sc->n_tris, p, J->s, J->t_eps, -1, -1) ||
                          brute_occluded(J->mtris, 2 * g->n_mods, p, J->s, J->t_eps, skip0, skip1);
                else
                    hit = bvh_occluded(&J->sc->bvh, p, J->s, J->t_eps, -1, -1) ||
                          bvh_occluded(J->mbvh, p, J->s, J->t_eps, skip0, skip1);
                int k = j * n + i;
                if (hit) { ++cnt; if (k < 64) bits |= 1ull << k; }
                if (g->want_mask) {
                    int msk = 1;
                    if (maskable) {
                        q.p = p;
                        if (g->brute)
                            msk = brute_masked(J->sc->tris, J->sc->n_tris, &q, -1, -1) ||
                                  brute_masked(J->mtris, 2 * g->n_mods, &q, skip0, skip1);
                        else
                            msk = bvh_masked(&J->sc->bvh, &q, t_lo, -1, -1) ||
                                  bvh_masked(J->mbvh, &q, t_lo, skip0, skip1);
                    }
                    if (msk && k < 64) mbits |= 1ull << k;
                }
            }
        }
        J->counts[cell] = cnt;
        if (J->bits) J->bits[cell] = bits;
        if (J->mbits) J->mbits[cell] = mbits;
    }
}

static void* worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (;;) {
        int64_t it = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (it >= J->n_items) break;
        eval_cell_row(J, J->item_mod[it], J->item_row[it]);
    }
    return NULL;
}

/*
 * Evaluate the generator over `n_eval_steps` steps (indices into the sun table)
 * and `n_eval` modules (indices into the module table; every module of the
 * generator still casts shadows).  Outputs are indexed by (eval step, eval cell)
 * or (eval step, eval module); cells of the evaluated modules are numbered in
 * the given module order, row-major (c = cv * cells_u + cu) within a module.
 *
 *   counts [S x C]   shaded samples per cell
 *   bits   [S x C]   shaded flag of sample k = j*n + i (n <= 8), or NULL
 *   mbits  [S x C]   parity-mask flag per sample (n <= 8), or NULL
 *   power, power_unshaded [S x M]   W at the maximum power point
 *   cos_inc [S x M]  cosine of incidence on the module
 *   delta   [S]      texel size of the step's light window (0 if the sun is down)
 *   cell_beam_loss [C]  sum over steps of DNI * max(0, cos) * f_c * dt   (Wh/m^2)
 *   energy, energy_unshaded [M]     sum over steps of P * dt (Wh)
 * Steps whose sun is at or below the horizon contribute nothing.
 * Returns 0, or -1 on invalid input.
 */
int pv3d_oracle_evaluate(void* scene_h,
                         int32_t n_mods, const float* mod_f, const int32_t* mod_i,
                         const int32_t* lay_off, const int32_t* lay_nsub, const int32_t* lay_sub,
                         int32_t n_trk, const float* pivots,
                         const double* sun, const float* dni, const float* dhi, const float* dt,
                         const float* poses,
                         int32_t n, int32_t map_res, double i_ref, double v_cell, double v_diode,
                         const int64_t* eval_steps, int64_t n_eval_steps,
                         const int32_t* eval_mods, int32_t n_eval,
                         int32_t want_mask, int32_t brute, int32_t n_threads,
                         int32_t* counts, uint64_t* bits, uint64_t* mbits,
                         double* power, double* power_unshaded, double* cos_inc, double* delta_out,
                         double* cell_beam_loss, double* energy, double* energy_unshaded)
{
    oscene_t* sc = (oscene_t*)scene_h;
    if (!sc || n < 1 || n_mods < 1 || map_res < 4 || n_eval < 1) return -1;
    ogen_t G = {n_mods, mod_f, mod_i, lay_off, lay_nsub, lay_sub, n_trk, pivots, sun, dni, dhi, dt,
                poses, n, map_res, i_ref, v_cell, v_diode, want_mask, brute};
    if (n_threads < 1) n_threads = 1;

    /* cell offsets of the evaluated modules and work items (one per cell row) */
    int64_t* cell_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_eval + 1));
    int64_t n_items = 0;
    cell_off[0] = 0;
    for (int32_t e = 0; e < n_eval; ++e) {
        const int32_t* mi = mod_i + 5 * (size_t)eval_mods[e];
        cell_off[e + 1] = cell_off[e] + (int64_t)mi[0] * mi[1];
        n_items += mi[1];
    }
    int64_t C = cell_off[n_eval];
    int32_t* item_mod = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_items);
    int32_t* item_row = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_items);
    {
        int64_t k = 0;
        for (int32_t e = 0; e < n_eval; ++e)
            for (int32_t r = 0; r < mod_i[5 * (size_t)eval_mods[e] + 1]; ++r) {
                item_mod[k] = e;
                item_row[k] = r;
                ++k;
            }
    }
    posed_t* posed = (posed_t*)malloc(sizeof(posed_t) * (size_t)n_mods);
    tri_t* mtris = (tri_t*)malloc(sizeof(tri_t) * 2 * (size_t)n_mods);
    double* gbuf = (double*)malloc(sizeof(double) * 4096);
    for (int32_t e = 0; e < n_eval; ++e) { energy[e] = 0; energy_unshaded[e] = 0; }
    for (int64_t c = 0; c < C; ++c) cell_beam_loss[c] = 0;

    /* scale of the scene for the ray offset */
    double scale = 1.0;
    for (int k = 0; k < 3; ++k)
        if (sc->n_tris) scale = fmax(scale, sc->hi[k] - sc->lo[k]);

    for (int64_t si = 0; si < n_eval_steps; ++si) {
        int64_t st = eval_steps[si];
        vec3 s = mk(sun[3 * st], sun[3 * st + 1], sun[3 * st + 2]);
        int32_t* cnt_s = counts + si * C;
        uint64_t* bits_s = bits ? bits + si * C : NULL;
        uint64_t* mbits_s = mbits ? mbits + si * C : NULL;
        if (!(s.z > 0.0)) {
            memset(cnt_s, 0, sizeof(int32_t) * (size_t)C);
            if (bits_s) memset(bits_s, 0, sizeof(uint64_t) * (size_t)C);
            if (mbits_s) memset(mbits_s, 0, sizeof(uint64_t) * (size_t)C);
            for (int32_t e = 0; e < n_eval; ++e) {
                power[si * n_eval + e] = 0; power_unshaded[si * n_eval + e] = 0;
                cos_inc[si * n_eval + e] = 0;
            }
            delta_out[si] = 0;
            continue;
        }
        /* pose every module, light window, module triangles */
        vec3 lu, lv;
        light_frame(s, &lu, &lv);
        double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        double mscale = scale;
        for (int32_t m = 0; m < n_mods; ++m) {
            pose_module(&G, m, st, &posed[m]);
            for (int k = 0; k < 4; ++k) {
                double pu = dot(posed[m].c[k], lu), pv = dot(posed[m].c[k], lv);
                umin = fmin(umin, pu); umax = fmax(umax, pu);
                vmin = fmin(vmin, pv); vmax = fmax(vmax, pv);
                mscale = fmax(mscale, fabs(posed[m].c[k].x));
                mscale = fmax(mscale, fabs(posed[m].c[k].y));
                mscale = fmax(mscale, fabs(posed[m].c[k].z));
            }
            mtris[2 * m].p[0] = posed[m].c[0];
            mtris[2 * m].p[1] = posed[m].c[1];
            mtris[2 * m].p[2] = posed[m].c[2];
            mtris[2 * m + 1].p[0] = posed[m].c[0];
            mtris[2 * m + 1].p[1] = posed[m].c[2];
            mtris[2 * m + 1].p[2] = posed[m].c[3];
        }
        double ext = fmax(umax - umin, vmax - vmin);
        double delta = ext / (double)(map_res - 2);
        delta_out[si] = delta;
        bvh_t mbvh;
        bvh_build(&mbvh, mtris, 2 * n_mods);

        job_t J;
        memset(&J, 0, sizeof(J));
        J.sc = sc; J.g = &G; J.posed = posed; J.mtris = mtris; J.mbvh = &mbvh;
        J.s = s; J.lu = lu; J.lv = lv; J.delta = delta;
        J.t_eps = 1e-9 * mscale;
        J.eps_h = 1e-9 * mscale;
        J.eval_mods = eval_mods; J.cell_off = cell_off; J.n_eval = n_eval;
        J.n_items = n_items; J.next = 0;
        J.counts = cnt_s; J.bits = bits_s; J.mbits = mbits_s;
        J.item_mod = item_mod;
        J.item_row = item_row;
        int nt = n_threads;
        if (nt > n_items) nt = (int)n_items;
        if (nt <= 1) {
            worker(&J);
        } else {
            pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
            for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, worker, &J);
            for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
            free(th);
        }
        bvh_free(&mbvh);

        /* reduction and PV model per evaluated module */
        for (int32_t e = 0; e < n_eval; ++e) {
            int32_t m = eval_mods[e];
            const int32_t* mi = mod_i + 5 * (size_t)m;
            int32_t ncell = mi[0] * mi[1];
            int32_t lay = mi[2];
            const int32_t* csub = lay_sub + lay_off[lay];
            double c = dot(posed[m].n, s);
            double beam = (double)dni[st] * fmax(0.0, c);
            double diff = (double)dhi[st] * (1.0 + posed[m].n.z) / 2.0;
            double* gs = ncell <= 2048 ? gbuf : (double*)malloc(sizeof(double) * 2 * (size_t)ncell);
            double* gu = gs + ncell;
            for (int32_t k = 0; k < ncell; ++k) {
                double fc = (double)cnt_s[cell_off[e] + k] / (double)(n * n);
                gs[k] = beam * (1.0 - fc) + diff;
                gu[k] = beam + diff;
                cell_beam_loss[cell_off[e] + k] += beam * fc * (double)dt[st];
            }
            double p = pv3d_oracle_module_pmpp(ncell, gs, csub, lay_nsub[lay], i_ref, v_cell, v_diode);
            double pu = pv3d_oracle_module_pmpp(ncell, gu, csub, lay_nsub[lay], i_ref, v_cell, v_diode);
            if (gs != gbuf) free(gs);
            power[si * n_eval + e] = p;
            power_unshaded[si * n_eval + e] = pu;
            cos_inc[si * n_eval + e] = c;
            energy[e] += p * (double)dt[st];
            energy_unshaded[e] += pu * (double)dt[st];
        }
    }
    free(cell_off); free(item_mod); free(item_row); free(posed); free(mtris); free(gbuf);
    return 0;
}

/*
 * PV model of Section 2 step 4 applied to given shaded-sample counts:
 * power[s * n_eval + e] for counts[s * C + cell] (cells of the evaluated
 * modules in order).  Used to check energy results cell count by cell count.
 */
int pv3d_oracle_power_from_counts(int32_t n_mods, const float* mod_f, const int32_t* mod_i,
                                  const int32_t* lay_off, const int32_t* lay_nsub, const int32_t* lay_sub,
                                  int32_t n_trk, const float* pivots, const double* sun, const float* dni,
                                  const float* dhi, const float* poses, int32_t n, double i_ref,
                                  double v_cell, double v_diode, const int64_t* eval_steps,
                                  int64_t n_eval_steps, const int32_t* eval_mods, int32_t n_eval,
                                  const int32_t* counts, double* power)
{
    ogen_t G;
    memset(&G, 0, sizeof(G));
    G.n_mods = n_mods; G.mod_f = mod_f; G.mod_i = mod_i; G.n_trk = n_trk; G.pivots = pivots;
    G.poses = poses; G.n = n;
    int64_t C = 0;
    for (int32_t e = 0; e < n_eval; ++e) C += (int64_t)mod_i[5 * (size_t)eval_mods[e]] * mod_i[5 * (size_t)eval_mods[e] + 1];
    double* g = (double*)malloc(sizeof(double) * 4096);
    for (int64_t si = 0; si < n_eval_steps; ++si) {
        int64_t st = eval_steps[si];
        vec3 s = mk(sun[3 * st], sun[3 * st + 1], sun[3 * st + 2]);
        int64_t c0 = 0;
        for (int32_t e = 0; e < n_eval; ++e) {
            int32_t m = eval_mods[e];
            const int32_t* mi = mod_i + 5 * (size_t)m;
            int32_t ncell = mi[0] * mi[1];
            if (!(s.z > 0.0) || ncell > 4096) {
                power[si * n_eval + e] = 0.0;
                c0 += ncell;
                continue;
            }
            posed_t P;
            pose_module(&G, m, st, &P);
            double c = dot(P.n, s);
            double beam = (double)dni[st] * fmax(0.0, c);
            double diff = (double)dhi[st] * (1.0 + P.n.z) / 2.0;
            for (int32_t k = 0; k < ncell; ++k) {
                double fc = (double)counts[si * C + c0 + k] / (double)(n * n);
                g[k] = beam * (1.0 - fc) + diff;
            }
            power[si * n_eval + e] = pv3d_oracle_module_pmpp(ncell, g, lay_sub + lay_off[mi[2]], lay_nsub[mi[2]],
                                                             i_ref, v_cell, v_diode);
            c0 += ncell;
        }
    }
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* series strings (Section 2: the generator's modules are wired in series     */
/* strings, Fig. 2)                                                           */
/* ------------------------------------------------------------------------- */
/*
 * One current I flows through every bypass substring of every module of a
 * string.  A substring k with current limit I_k and voltage V_k (its cells in
 * series, as in pv3d_oracle_module_pmpp) delivers V_k while I <= I_k and costs
 * v_diode through its bypass diode above.  The string's
 * P(I) = I * (sum_{k: I_k >= I} V_k - v_diode * #{k: I_k < I}) is linear
 * between consecutive I_k, so its maximum power point is the best of the I_k
 * (and 0).  The module model is the one-module string.
 */
double pv3d_oracle_series_pmpp(int32_t n_sub, const double* ik, const double* vk, double v_diode)
{
    double best = 0.0;
    for (int32_t k = 0; k < n_sub; ++k) {
        double cur = ik[k];
        double volt = 0.0;
        for (int32_t j = 0; j < n_sub; ++j) volt += (ik[j] >= cur) ? vk[j] : -v_diode;
        double p = cur * volt;
        if (p > best) best = p;
    }
    return best;
}

/*
 * Strings in parallel at one maximum power point tracker (the inverter's
 * input: Section 2's generator of strings, Fig. 2).  One voltage V is across
 * every string; string s delivers the largest current I at which its voltage
 * V_s(I) = sum_{k: I_k >= I} V_k - v_diode * #{k: I_k < I} still reaches V.
 * V_s is a non-increasing step function of I whose steps are at the
 * substring currents, so string s's current at V is the largest I_k of its
 * substrings with V_s(I_k) >= V (0 if none), and P(V) = V * sum_s I_s(V) is
 * linear in V between the voltages V_s(I_k): its maximum is the best of
 * those voltages.  String s owns substrings [str_off[s], str_off[s + 1]).
 */
double pv3d_oracle_parallel_pmpp(int32_t n_str, const int32_t* str_off, const double* ik, const double* vk,
                                 double v_diode)
{
    int32_t n_all = str_off[n_str];
    double* w = (double*)malloc(sizeof(double) * (size_t)(n_all > 0 ? n_all : 1));
    for (int32_t s = 0; s < n_str; ++s)
        for (int32_t k = str_off[s]; k < str_off[s + 1]; ++k) {
            double v = 0.0;
            for (int32_t j = str_off[s]; j < str_off[s + 1]; ++j) v += (ik[j] >= ik[k]) ? vk[j] : -v_diode;
            w[k] = v;  /* string s's voltage at current ik[k] */
        }
    double best = 0.0;
    for (int32_t c = 0; c < n_all; ++c) {
        double V = w[c];
        if (!(V > 0.0)) continue;
        double cur = 0.0;
        for (int32_t s = 0; s < n_str; ++s) {
            double is = 0.0;
            for (int32_t k = str_off[s]; k < str_off[s + 1]; ++k)
                if (w[k] >= V && ik[k] > is) is = ik[k];
            cur += is;
        }
        if (V * cur > best) best = V * cur;
    }
    free(w);
    return best;
}

/* Current limit and voltage of each substring of one module from its cell
 * irradiances g (W/m^2): written to ik[0..n_sub), vk[0..n_sub). */
static void module_substrings(int32_t n_cells, const double* g, const int32_t* cell_sub, int32_t n_sub,
                              double i_ref, double v_cell, double* ik, double* vk)
{
    for (int32_t k = 0; k < n_sub; ++k) { ik[k] = INFINITY; vk[k] = 0.0; }
    for (int32_t c = 0; c < n_cells; ++c) {
        int32_t k = cell_sub[c];
        double ic = i_ref * g[c] / 1000.0;
        if (ic < ik[k]) ik[k] = ic;
        vk[k] += v_cell;
    }
}

/*
 * String powers for given shaded-sample counts: power[s * n_str + q] and
 * power_unshaded[s * n_str + q] of string q, where mod_string[m] = q names the
 * string of module m, and counts[s * C + cell] holds every module's cells in
 * module order.  A step with the sun at or below the horizon gives 0.  With
 * str_array (string q in parallel array str_array[q] < n_arr) and apower /
 * apower_u non-NULL, also the powers of the arrays of strings in parallel,
 * apower[s * n_arr + a].
 */
int pv3d_oracle_string_power_from_counts(int32_t n_mods, const float* mod_f, const int32_t* mod_i,
                                         const int32_t* lay_off, const int32_t* lay_nsub, const int32_t* lay_sub,
                                         int32_t n_trk, const float* pivots, const double* sun, const float* dni,
                                         const float* dhi, const float* poses, int32_t n, double i_ref,
                                         double v_cell, double v_diode, const int64_t* eval_steps,
                                         int64_t n_eval_steps, const int32_t* mod_string, int32_t n_str,
                                         const int32_t* counts, double* power, double* power_unshaded,
                                         const int32_t* str_array, int32_t n_arr, double* apower, double* apower_u)
{
    ogen_t G;
    memset(&G, 0, sizeof(G));
    G.n_mods = n_mods; G.mod_f = mod_f; G.mod_i = mod_i; G.n_trk = n_trk; G.pivots = pivots;
    G.poses = poses; G.n = n;
    int64_t C = 0, n_sub_all = 0;
    int64_t* cell0 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_mods + 1));
    for (int32_t m = 0; m < n_mods; ++m) {
        cell0[m] = C;
        C += (int64_t)mod_i[5 * (size_t)m] * mod_i[5 * (size_t)m + 1];
        n_sub_all += lay_nsub[mod_i[5 * (size_t)m + 2]];
    }
    cell0[n_mods] = C;
    /* substrings of each string, gathered module by module */
    double* ik = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
    double* vk = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
    double* iu = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
    int64_t* str_fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_str + 1));
    int64_t* str_base = (int64_t*)calloc((size_t)(n_str + 1), sizeof(int64_t));
    for (int32_t m = 0; m < n_mods; ++m) str_base[mod_string[m] + 1] += lay_nsub[mod_i[5 * (size_t)m + 2]];
    for (int32_t q = 0; q < n_str; ++q) str_base[q + 1] += str_base[q];
    double* g = (double*)malloc(sizeof(double) * 2048);
    double* gu = (double*)malloc(sizeof(double) * 2048);
    double tik[64], tvk[64], tiu[64], tvu[64];
    for (int64_t si = 0; si < n_eval_steps; ++si) {
        int64_t st = eval_steps[si];
        vec3 s = mk(sun[3 * st], sun[3 * st + 1], sun[3 * st + 2]);
        for (int32_t q = 0; q < n_str; ++q) str_fill[q] = str_base[q];
        for (int32_t m = 0; m < n_mods; ++m) {
            const int32_t* mi = mod_i + 5 * (size_t)m;
            int32_t ncell = mi[0] * mi[1], lay = mi[2], ns = lay_nsub[lay];
            posed_t P;
            pose_module(&G, m, st, &P);
            double c = dot(P.n, s);
            double beam = s.z > 0.0 ? (double)dni[st] * fmax(0.0, c) : 0.0;
            double diff = s.z > 0.0 ? (double)dhi[st] * (1.0 + P.n.z) / 2.0 : 0.0;
            for (int32_t k = 0; k < ncell; ++k) {
                double fc = (double)counts[si * C + cell0[m] + k] / (double)(n * n);
                g[k] = beam * (1.0 - fc) + diff;
                gu[k] = beam + diff;
            }
            module_substrings(ncell, g, lay_sub + lay_off[lay], ns, i_ref, v_cell, tik, tvk);
            module_substrings(ncell, gu, lay_sub + lay_off[lay], ns, i_ref, v_cell, tiu, tvu);
            int64_t f = str_fill[mod_string[m]];
            for (int32_t k = 0; k < ns; ++k) { ik[f + k] = tik[k]; vk[f + k] = tvk[k]; iu[f + k] = tiu[k]; }
            str_fill[mod_string[m]] = f + ns;
        }
        for (int32_t q = 0; q < n_str; ++q) {
            int64_t b = str_base[q], e = str_base[q + 1];
            power[si * n_str + q] = pv3d_oracle_series_pmpp((int32_t)(e - b), ik + b, vk + b, v_diode);
            power_unshaded[si * n_str + q] = pv3d_oracle_series_pmpp((int32_t)(e - b), iu + b, vk + b, v_diode);
        }
        if (str_array && apower && apower_u) {
            /* each array: its strings' substrings gathered, string by string */
            double* gi = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
            double* gu = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
            double* gv = (double*)malloc(sizeof(double) * (size_t)(n_sub_all + 1));
            int32_t* off = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_str + 1));
            for (int32_t a = 0; a < n_arr; ++a) {
                int32_t ns = 0, nk = 0;
                off[0] = 0;
                for (int32_t q = 0; q < n_str; ++q) {
                    if (str_array[q] != a) continue;
                    for (int64_t k = str_base[q]; k < str_base[q + 1]; ++k) {
                        gi[nk] = ik[k]; gu[nk] = iu[k]; gv[nk] = vk[k];
                        ++nk;
                    }
                    off[++ns] = nk;
                }
                apower[si * n_arr + a] = pv3d_oracle_parallel_pmpp(ns, off, gi, gv, v_diode);
                apower_u[si * n_arr + a] = pv3d_oracle_parallel_pmpp(ns, off, gu, gv, v_diode);
            }
            free(gi); free(gu); free(gv); free(off);
        }
    }
    free(cell0); free(ik); free(vk); free(iu); free(str_fill); free(str_base); free(g); free(gu);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* sun table (the inputs of steps 3-4: sun positions and irradiance over the  */
/* simulated period -- the paper takes TMY data, measured series or a        */
/* clear-sky model without naming one)                                        */
/* ------------------------------------------------------------------------- */
/*
 * Reading: solar time without longitude correction or equation of time; the
 * declination of Cooper (1969), delta = 23.45 deg * sin(360 deg * (284 + n) / 365)
 * on day n; the hour angle omega = 15 deg * (t - 12) at solar hour t.  The unit
 * vector toward the sun, east-north-up, is the rotation of the equatorial
 * direction (cos delta cos omega, cos delta sin omega, sin delta) to the site:
 *   east  = -cos(delta) sin(omega)
 *   north =  sin(delta) cos(phi) - cos(delta) cos(omega) sin(phi)
 *   up    =  sin(delta) sin(phi) + cos(delta) cos(omega) cos(phi).
 * Beam irradiance of Meinel & Meinel (1976), DNI = 1353 * 0.7^(AM^0.678) W/m^2,
 * with the air mass of Kasten & Young (1989),
 * AM = 1 / (cos z + 0.50572 (96.07995 - z)^-1.6364), z the zenith angle in
 * degrees; diffuse DHI = dhi_fraction * DNI; both 0 with the sun at or below
 * the horizon.  Steps at t = 0, step_h, 2 step_h, ... (t < 24) of days
 * day_first .. day_first + n_days - 1; with daylight_only only the steps with
 * up > 0 are kept.  Returns the number of steps (xyz, dni, dhi may be NULL to
 * count them).
 */
int64_t pv3d_oracle_sun_table(double lat_deg, int32_t day_first, int32_t n_days, double step_h,
                              int32_t daylight_only, double dhi_fraction, double* xyz, double* dni, double* dhi)
{
    const double deg = M_PI / 180.0;
    const double phi = lat_deg * deg;
    int64_t per_day = 0;
    while (per_day * step_h < 24.0 - 1e-9) ++per_day;
    int64_t out = 0;
    for (int32_t d = 0; d < n_days; ++d) {
        double n = (double)(day_first + d);
        double delta = 23.45 * deg * sin(360.0 * deg * (284.0 + n) / 365.0);
        for (int64_t k = 0; k < per_day; ++k) {
            double t = (double)k * step_h;
            double omega = 15.0 * deg * (t - 12.0);
            double e = -cos(delta) * sin(omega);
            double nn = sin(delta) * cos(phi) - cos(delta) * cos(omega) * sin(phi);
            double u = sin(delta) * sin(phi) + cos(delta) * cos(omega) * cos(phi);
            double len = sqrt(e * e + nn * nn + u * u);
            e /= len; nn /= len; u /= len;
            if (daylight_only && !(u > 0.0)) continue;
            double b = 0.0;
            if (u > 0.0) {
                double z = acos(u) / deg;
                double am = 1.0 / (u + 0.50572 * pow(96.07995 - z, -1.6364));
                b = 1353.0 * pow(0.7, pow(am, 0.678));
            }
            if (xyz) { xyz[3 * out] = e; xyz[3 * out + 1] = nn; xyz[3 * out + 2] = u; }
            if (dni) dni[out] = b;
            if (dhi) dhi[out] = dhi_fraction * b;
            ++out;
        }
    }
    return out;
}

/* Sample positions of one module at one step (for tests): xyz[cells*n*n*3] in
 * cell order, then sample order k = j*n + i. */
int pv3d_oracle_samples(int32_t n_mods, const float* mod_f, const int32_t* mod_i, int32_t n_trk,
                        const float* pivots, const float* poses, int64_t step, int32_t module,
                        int32_t n, double* xyz)
{
    ogen_t G;
    memset(&G, 0, sizeof(G));
    G.n_mods = n_mods; G.mod_f = mod_f; G.mod_i = mod_i; G.n_trk = n_trk; G.pivots = pivots;
    G.poses = poses; G.n = n;
    if (module < 0 || module >= n_mods) return -1;
    posed_t P;
    pose_module(&G, module, step, &P);
    const int32_t* mi = mod_i + 5 * (size_t)module;
    double pitch = mod_f[10 * (size_t)module + 9];
    int64_t k = 0;
    for (int32_t cv = 0; cv < mi[1]; ++cv)
        for (int32_t cu = 0; cu < mi[0]; ++cu)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double a = (cu + (i + 0.5) / n) * pitch, b = (cv + (j + 0.5) / n) * pitch;
                    vec3 p = add(add(P.o, scl(P.u, a)), scl(P.v, b));
                    xyz[3 * k] = p.x; xyz[3 * k + 1] = p.y; xyz[3 * k + 2] = p.z;
                    ++k;
                }
    return 0;
}

/* Posed unit normal of one module (for tests). */
int pv3d_oracle_module_normal(int32_t n_mods, const float* mod_f, const int32_t* mod_i, int32_t n_trk,
                              const float* pivots, const float* poses, int64_t step, int32_t module,
                              double* nrm)
{
    ogen_t G;
    memset(&G, 0, sizeof(G));
    G.n_mods = n_mods; G.mod_f = mod_f; G.mod_i = mod_i; G.n_trk = n_trk; G.pivots = pivots;
    G.poses = poses;
    if (module < 0 || module >= n_mods) return -1;
    posed_t P;
    pose_module(&G, module, step, &P);
    nrm[0] = P.n.x; nrm[1] = P.n.y; nrm[2] = P.n.z;
    return 0;
}

/* Ray query on a scene alone (for tests): flags[i] = 1 iff the ray from o_i
 * along d_i meets a triangle at t > t_min. */
int pv3d_oracle_rays(void* scene_h, const double* o, const double* d, int64_t n_rays, double t_min,
                     int32_t brute, uint8_t* flags)
{
    oscene_t* sc = (oscene_t*)scene_h;
    if (!sc) return -1;
    for (int64_t r = 0; r < n_rays; ++r) {
        vec3 oo = mk(o[3 * r], o[3 * r + 1], o[3 * r + 2]);
        vec3 dd = mk(d[3 * r], d[3 * r + 1], d[3 * r + 2]);
        flags[r] = (uint8_t)(brute ? brute_occluded(sc->tris, sc->n_tris, oo, dd, t_min, -1, -1)
                                   : bvh_occluded(&sc->bvh, oo, dd, t_min, -1, -1));
    }
    return 0;
}
