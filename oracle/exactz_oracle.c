/*
 * exactz_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow CPU statement of the EXaCTz bounded-iteration correction
 * (Li et al., "EXaCTz", Algorithm 1 with the EG constraints of Sec. 4.2 and the
 * reformulated event constraints of Sec. 4.3, or the saddle-ordering and the
 * original merge / split event constraints of Sec. 4.2).  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library: the mesh is re-derived here
 * from explicit tetrahedra, neighbour searches compare values one pair at a
 * time, and link components are found by a plain graph search.
 *
 * Readings of the paper fixed here (the paper is silent on them):
 *  - Mesh: the PL field of Sec. 3 lives on the Freudenthal (Kuhn) triangulation
 *    of the vertex grid: every unit cube is cut into six tetrahedra, one per
 *    permutation of the axes, each a monotone lattice path from the cube's low
 *    corner to its high corner.  Two vertices are neighbours iff they share a
 *    tetrahedron.  Out-of-domain vertices do not exist (no periodicity).
 *  - Order (Sec. 3.3 footnote, simulation of simplicity): u precedes v in field
 *    h iff h_u < h_v, or h_u == h_v and u < v (IEEE compare, so -0 == +0).
 *  - Steepest neighbours (Sec. 3.1, Sec. 4.2): up_h(i) / down_h(i) are the
 *    largest / smallest vertex of the closed neighbourhood N(i) + {i}.
 *  - Classification (Sec. 3.2 Step 1): with L (U) the neighbours below (above)
 *    i, cL (cU) = number of connected components of the link of i restricted
 *    to L (U).  minimum iff cL = 0; else maximum iff cU = 0; else join saddle if
 *    cL >= 2, split saddle if cU >= 2 (both may hold); otherwise regular.
 *  - One iteration is synchronous (Jacobi): the request set R is formed from
 *    the current g, then every requested vertex is edited at most once
 *    (Sec. 4.4 proof: "at most once per iteration").  Rules:
 *      R1 (Sec. 4.2, EG constraints): for every vertex i, if up_g(i) != up_f(i)
 *         request up_g(i); if down_g(i) != down_f(i) request down_f(i).
 *      R2 (Sec. 4.2, saddles): for every i that is a saddle in f or in g and
 *         every neighbour j, if the order of (j, i) differs between f and g,
 *         request whichever of i, j is lower in f.
 *      R3 (Sec. 4.3, reformulated event constraints, which subsume the
 *         saddle-ordering constraint C2): with o the critical points of f sorted
 *         by the f-order, for each adjacent pair (o[p], o[p+1]) whose g-order is
 *         reversed, request o[p].
 *  - Edit (Sec. 3.3): Delta = fl(xi / N) in binary32; floor_i = fl(f_i - xi).
 *    With k_i edits so far: if k_i < N, t = fl(g_i - Delta); if t < floor_i
 *    then g_i = floor_i, k_i = N + 1, else g_i = t, k_i += 1.  If k_i == N the
 *    "more than N edits" rule stores the lossless bound: g_i = floor_i,
 *    k_i = N + 1.  A vertex with k_i == N + 1 is pinned and never changes.
 *  - Termination (Algorithm 1's "S is empty"): let R* = requested vertices that
 *    are not pinned.  Stop when R* is empty: status CONVERGED if R is empty,
 *    else STUCK (requests remain only on pinned vertices, which happens only
 *    through float ties at the floors).  Stop with ITER_LIMIT when R* is not
 *    empty after max_iters edit passes.  iterations = edit passes executed;
 *    residual = |R| of the last check.
 *
 * Original event constraints (Sec. 4.2 "Saddle Ordering Constraints" and
 * "Merge and Split Event Constraints"; oracle_correct_events), used instead of
 * R3:
 *      C2: with so the saddles of f sorted by the f-order, for each adjacent
 *          pair (so[q], so[q+1]) whose g-order is reversed, request so[q].
 *      C3: the extremum graph of f links a join saddle s to minimum m when
 *          the steepest-descent path (down_f repeatedly) from some neighbour
 *          of s below s ends at m (Sec. 3.2 Step 1).  Extremum Graph Pairing
 *          selects the largest of the minima linked to s.  If the largest in g
 *          (among the same minima) differs from the one in f, request the one
 *          selected in g (it lies below the f-selection in f).  Split saddles
 *          symmetrically: steepest-ascent paths (up_f) from the neighbours above
 *          a split saddle reach its maxima, EGP selects the smallest maximum, and a
 *          differing g-selection requests the f-selection (the lower of the two
 *          in f).  A saddle whose paths reach a single extremum has no event.
 *
 * Worklist mode evaluates R1/R2 only at vertices whose closed neighbourhood
 * holds a vertex edited in the previous pass, and R3 only on pairs touching an
 * edited critical point.  Every rule at i reads and targets only N(i) + {i}
 * (or its pair), so an unevaluated checker would re-issue last pass's request,
 * whose target was either edited (then the checker is evaluated) or pinned; the
 * set R* is therefore identical.  The residual count is taken by a full sweep.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_CONVERGED 1
#define OR_STUCK 2
#define OR_ITER_LIMIT 3
#define OR_EINVAL (-1)
#define OR_ENONFINITE (-2)
#define OR_EBOUND (-3)
#define OR_ENOMEM (-4)

#define T_MIN 1
#define T_MAX 2
#define T_JOIN 4
#define T_SPLIT 8

/* ------------------------------------------------------------------ mesh */

static int g_ready = 0;
static int g_noff = 0;           /* number of neighbour offsets found     */
static int g_off[32][3];         /* offset of neighbour slot s            */
static unsigned char g_link[32][32]; /* link edge between slots a and b   */

static int find_off(const int d[3])
{
    for (int s = 0; s < g_noff; s++)
        if (g_off[s][0] == d[0] && g_off[s][1] == d[1] && g_off[s][2] == d[2])
            return s;
    return -1;
}

static int add_off(const int d[3])
{
    int s = find_off(d);
    if (s >= 0) return s;
    g_off[g_noff][0] = d[0];
    g_off[g_noff][1] = d[1];
    g_off[g_noff][2] = d[2];
    return g_noff++;
}

/* Enumerate the 6 tetrahedra of each of the 8 unit cubes that have the origin
 * as a corner.  Every other vertex of a tetrahedron holding the origin is a
 * neighbour; every edge of such a tetrahedron not touching the origin is an
 * edge of the origin's link. */
static void derive_mesh(void)
{
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                   {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    if (g_ready) return;
    g_noff = 0;
    memset(g_link, 0, sizeof(g_link));
    for (int s = 0; s < 8; s++) {
        int c[3] = {-(s & 1), -((s >> 1) & 1), -((s >> 2) & 1)};
        for (int t = 0; t < 6; t++) {
            int v[4][3];
            v[0][0] = c[0]; v[0][1] = c[1]; v[0][2] = c[2];
            for (int m = 1; m < 4; m++) {
                v[m][0] = v[m - 1][0]; v[m][1] = v[m - 1][1]; v[m][2] = v[m - 1][2];
                v[m][perm[t][m - 1]] += 1;
            }
            int at = -1;
            for (int m = 0; m < 4; m++)
                if (v[m][0] == 0 && v[m][1] == 0 && v[m][2] == 0) at = m;
            if (at < 0) continue;
            int sl[4] = {-1, -1, -1, -1};
            for (int m = 0; m < 4; m++)
                if (m != at) sl[m] = add_off(v[m]);
            for (int a = 0; a < 4; a++)
                for (int b = a + 1; b < 4; b++)
                    if (a != at && b != at) {
                        g_link[sl[a]][sl[b]] = 1;
                        g_link[sl[b]][sl[a]] = 1;
                    }
        }
    }
    g_ready = 1;
}

/* Export the derived mesh: offsets (3 ints each) and link edges (slot pairs). */
int oracle_mesh(int *offsets_out, int *n_off, int *edges_out, int *n_edges)
{
    derive_mesh();
    *n_off = g_noff;
    for (int s = 0; s < g_noff; s++)
        for (int a = 0; a < 3; a++) offsets_out[3 * s + a] = g_off[s][a];
    int e = 0;
    for (int a = 0; a < g_noff; a++)
        for (int b = a + 1; b < g_noff; b++)
            if (g_link[a][b]) {
                edges_out[2 * e] = a;
                edges_out[2 * e + 1] = b;
                e++;
            }
    *n_edges = e;
    return 0;
}

typedef struct {
    int64_t nx, ny, nz, n;
} grid_t;

/* In-domain neighbours of p: vertex ids and their slots. */
static int neighbours(const grid_t *G, int64_t p, int64_t *nb, int *slot)
{
    int64_t x = p % G->nx, y = (p / G->nx) % G->ny, z = p / (G->nx * G->ny);
    int c = 0;
    for (int s = 0; s < g_noff; s++) {
        int64_t X = x + g_off[s][0], Y = y + g_off[s][1], Z = z + g_off[s][2];
        if (X < 0 || Y < 0 || Z < 0 || X >= G->nx || Y >= G->ny || Z >= G->nz) continue;
        nb[c] = X + G->nx * (Y + G->ny * Z);
        slot[c] = s;
        c++;
    }
    return c;
}

/* a precedes b in field h (simulation of simplicity by vertex index). */
static int prec(const float *h, int64_t a, int64_t b)
{
    return h[a] < h[b] || (h[a] == h[b] && a < b);
}

/* Number of connected components of the link restricted to the members m[]
 * (m[j] != 0) of the neighbour list, by repeated depth-first search. */
static int components(const int *slot, int cnt, const int *member)
{
    int seen[32] = {0};
    int stack[32];
    int comps = 0;
    for (int a = 0; a < cnt; a++) {
        if (!member[a] || seen[a]) continue;
        comps++;
        int sp = 0;
        stack[sp++] = a;
        seen[a] = 1;
        while (sp) {
            int u = stack[--sp];
            for (int b = 0; b < cnt; b++)
                if (member[b] && !seen[b] && g_link[slot[u]][slot[b]]) {
                    seen[b] = 1;
                    stack[sp++] = b;
                }
        }
    }
    return comps;
}

static void classify_vertex(const grid_t *G, const float *h, int64_t p,
                            int64_t *up, int64_t *down, uint8_t *type)
{
    int64_t nb[32];
    int slot[32];
    int cnt = neighbours(G, p, nb, slot);
    int64_t bu = p, bd = p;
    for (int j = 0; j < cnt; j++) {
        if (prec(h, bu, nb[j])) bu = nb[j];
        if (prec(h, nb[j], bd)) bd = nb[j];
    }
    *up = bu;
    *down = bd;
    int inL[32], inU[32];
    for (int j = 0; j < cnt; j++) {
        inL[j] = prec(h, nb[j], p);
        inU[j] = !inL[j];
    }
    int cL = components(slot, cnt, inL);
    int cU = components(slot, cnt, inU);
    uint8_t t = 0;
    if (cL == 0) t = T_MIN;
    else if (cU == 0) t = T_MAX;
    else {
        if (cL >= 2) t |= T_JOIN;
        if (cU >= 2) t |= T_SPLIT;
    }
    *type = t;
}

static int dims_ok(int64_t nx, int64_t ny, int64_t nz)
{
    return nx >= 1 && ny >= 1 && nz >= 1 && nx * ny * nz >= 2;
}

/* Classification of every vertex of h: steepest up/down vertex and type. */
int oracle_classify(const float *h, int64_t nx, int64_t ny, int64_t nz,
                    int64_t *up, int64_t *down, uint8_t *type)
{
    if (!dims_ok(nx, ny, nz)) return OR_EINVAL;
    derive_mesh();
    grid_t G = {nx, ny, nz, nx * ny * nz};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < G.n; p++) classify_vertex(&G, h, p, &up[p], &down[p], &type[p]);
    return 0;
}

/* Sorting the critical points by the f-order.  qsort has no context argument,
 * so the field is passed through a file-scope pointer (single caller at a time). */
static const float *g_sort_field;
static int cmp_order(const void *a, const void *b)
{
    int64_t u = *(const int64_t *)a, v = *(const int64_t *)b;
    if (u == v) return 0;
    return prec(g_sort_field, u, v) ? -1 : 1;
}

static int64_t cp_order(const float *f, const uint8_t *type, int64_t n, int64_t *o)
{
    int64_t c = 0;
    for (int64_t p = 0; p < n; p++)
        if (type[p] != 0) o[c++] = p;
    g_sort_field = f;
    qsort(o, (size_t)c, sizeof(int64_t), cmp_order);
    return c;
}

/* Critical points of f in ascending f-order; returns their count. */
int64_t oracle_cp_order(const float *f, int64_t nx, int64_t ny, int64_t nz, int64_t *order_out)
{
    if (!dims_ok(nx, ny, nz)) return OR_EINVAL;
    int64_t n = nx * ny * nz;
    int64_t *up = malloc(sizeof(int64_t) * n), *dn = malloc(sizeof(int64_t) * n);
    uint8_t *ty = malloc(n);
    if (!up || !dn || !ty) { free(up); free(dn); free(ty); return OR_ENOMEM; }
    oracle_classify(f, nx, ny, nz, up, dn, ty);
    int64_t c = cp_order(f, ty, n, order_out);
    free(up); free(dn); free(ty);
    return c;
}

/* ------------------------------------------------------------ correction */

typedef struct {
    grid_t G;
    const float *f;
    int64_t *upf, *dnf;
    uint8_t *tyf;
    int64_t *o;       /* critical points of f, sorted by the f-order */
    int64_t ncp;
    int64_t *rank;    /* position of a critical point in o, -1 otherwise */
    /* increasing edits (inc = 1): every rule raises the vertex that must be higher */
    int inc;
    /* original event constraints (events = 1) */
    int events;
    int64_t *so;      /* saddles of f, sorted by the f-order */
    int64_t nso;
    int64_t *ev_ext;  /* per sorted saddle q, up to EV_MAX extrema: minima of a join saddle, then maxima of a split */
    uint8_t *ev_nmin, *ev_nmax;
    int64_t *sel_min, *sel_max;  /* per sorted saddle: EGP selection in f, -1 if none */
} ctx_t;

#define EV_MAX 14 /* the neighbours of a vertex */

static void mark(uint8_t *req, int64_t x)
{
#pragma omp atomic write
    req[x] = 1;
}

/* Evaluate rules R1 and R2 at vertex p for the current g. */
static void check_vertex(const ctx_t *C, const float *g, int64_t p, uint8_t *req)
{
    int64_t upg, dng;
    uint8_t tyg;
    classify_vertex(&C->G, g, p, &upg, &dng, &tyg);
    if (upg != C->upf[p]) mark(req, C->inc ? C->upf[p] : upg);
    if (dng != C->dnf[p]) mark(req, C->inc ? dng : C->dnf[p]);
    int saddle_f = (C->tyf[p] & (T_JOIN | T_SPLIT)) != 0;
    int saddle_g = (tyg & (T_JOIN | T_SPLIT)) != 0;
    if (saddle_f || saddle_g) {
        int64_t nb[32];
        int slot[32];
        int cnt = neighbours(&C->G, p, nb, slot);
        for (int j = 0; j < cnt; j++) {
            int below_f = prec(C->f, nb[j], p);
            int below_g = prec(g, nb[j], p);
            if (below_f != below_g) mark(req, (below_f != C->inc) ? nb[j] : p);
        }
    }
}

/* Evaluate rule R3 on the sorted pair (o[q], o[q+1]). */
static void check_pair(const ctx_t *C, const float *g, int64_t q, uint8_t *req)
{
    int64_t a = C->o[q], b = C->o[q + 1];
    if (prec(g, b, a)) mark(req, C->inc ? b : a);
}

/* C2 on the sorted saddle pair (so[q], so[q+1]). */
static void check_saddle_pair(const ctx_t *C, const float *g, int64_t q, uint8_t *req)
{
    int64_t a = C->so[q], b = C->so[q + 1];
    if (prec(g, b, a)) mark(req, C->inc ? b : a);
}

/* C3 at the sorted saddle so[q]: the EGP selection among its connected extrema in g. */
static void check_events(const ctx_t *C, const float *g, int64_t q, uint8_t *req)
{
    const int64_t *e = C->ev_ext + q * EV_MAX;
    int nm = C->ev_nmin[q], nx = C->ev_nmax[q];
    if (C->sel_min[q] >= 0) {
        int64_t best = e[0];
        for (int j = 1; j < nm; j++)
            if (prec(g, best, e[j])) best = e[j];
        if (best != C->sel_min[q]) mark(req, C->inc ? C->sel_min[q] : best);
    }
    if (C->sel_max[q] >= 0) {
        int64_t best = e[nm];
        for (int j = 1; j < nx; j++)
            if (prec(g, e[nm + j], best)) best = e[nm + j];
        if (best != C->sel_max[q]) mark(req, C->inc ? best : C->sel_max[q]);
    }
}

static int64_t count_set(const uint8_t *req, int64_t n)
{
    int64_t c = 0;
    for (int64_t p = 0; p < n; p++) c += req[p] != 0;
    return c;
}

/* Full sweep: every vertex and every pair; returns |R|. */
static int64_t check_full(const ctx_t *C, const float *g, uint8_t *req)
{
    memset(req, 0, (size_t)C->G.n);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t p = 0; p < C->G.n; p++) check_vertex(C, g, p, req);
    if (!C->events) {
        const int64_t npairs = C->ncp - 1;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < npairs; q++) check_pair(C, g, q, req);
    } else {
        const int64_t npairs = C->nso - 1;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < npairs; q++) check_saddle_pair(C, g, q, req);
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < C->nso; q++) check_events(C, g, q, req);
    }
    return count_set(req, C->G.n);
}

/* Terminal extremum of the integral path from v along the steepest links.
 * end[] (-1 = not known yet) remembers the terminal of every vertex walked, so
 * that paths shared by many saddles are walked once. */
static int64_t path_end(const int64_t *step, int64_t *end, int64_t v)
{
    int64_t u = v;
    while (end[u] < 0 && step[u] != u) u = step[u];
    const int64_t m = end[u] >= 0 ? end[u] : u;
    for (int64_t w = v; end[w] < 0; w = step[w]) {
        end[w] = m;
        if (w == u) break;
    }
    return m;
}

/* The extremum graph of f at its saddles and its EGP selections (C3), and the
 * sorted saddles (C2). */
static int setup_events(ctx_t *C)
{
    const int64_t n = C->G.n;
    int64_t nso = 0;
    for (int64_t q = 0; q < C->ncp; q++) nso += (C->tyf[C->o[q]] & (T_JOIN | T_SPLIT)) != 0;
    const size_t m = (size_t)(nso > 0 ? nso : 1);
    C->so = malloc(sizeof(int64_t) * m);
    C->ev_ext = malloc(sizeof(int64_t) * m * EV_MAX);
    C->ev_nmin = calloc(m, 1);
    C->ev_nmax = calloc(m, 1);
    C->sel_min = malloc(sizeof(int64_t) * m);
    C->sel_max = malloc(sizeof(int64_t) * m);
    if (!C->so || !C->ev_ext || !C->ev_nmin || !C->ev_nmax || !C->sel_min || !C->sel_max) return OR_ENOMEM;
    C->nso = 0;
    for (int64_t q = 0; q < C->ncp; q++)
        if (C->tyf[C->o[q]] & (T_JOIN | T_SPLIT)) C->so[C->nso++] = C->o[q];
    for (int64_t q = 0; q < nso; q++) C->sel_min[q] = C->sel_max[q] = -1;
    int64_t *end_dn = malloc(sizeof(int64_t) * n), *end_up = malloc(sizeof(int64_t) * n);
    if (!end_dn || !end_up) {
        free(end_dn);
        free(end_up);
        return OR_ENOMEM;
    }
    for (int64_t p = 0; p < n; p++) end_dn[p] = end_up[p] = -1;
    for (int64_t q = 0; q < C->nso; q++) {
        const int64_t s = C->so[q];
        int64_t nb[32];
        int slot[32];
        const int cnt = neighbours(&C->G, s, nb, slot);
        int64_t *e = C->ev_ext + q * EV_MAX;
        int ne = 0;
        if (C->tyf[s] & T_JOIN) {
            for (int j = 0; j < cnt; j++) {
                if (!prec(C->f, nb[j], s)) continue;
                const int64_t m = path_end(C->dnf, end_dn, nb[j]);
                int dup = 0;
                for (int i = 0; i < ne; i++) dup |= e[i] == m;
                if (!dup) e[ne++] = m;
            }
            C->ev_nmin[q] = (uint8_t)ne;
            if (ne >= 2) {
                int64_t best = e[0];
                for (int i = 1; i < ne; i++)
                    if (prec(C->f, best, e[i])) best = e[i];
                C->sel_min[q] = best;
            }
        }
        const int nm = ne;
        if (C->tyf[s] & T_SPLIT) {
            for (int j = 0; j < cnt; j++) {
                if (!prec(C->f, s, nb[j])) continue;
                const int64_t m = path_end(C->upf, end_up, nb[j]);
                int dup = 0;
                for (int i = nm; i < ne; i++) dup |= e[i] == m;
                if (!dup) e[ne++] = m;
            }
            C->ev_nmax[q] = (uint8_t)(ne - nm);
            if (ne - nm >= 2) {
                int64_t best = e[nm];
                for (int i = nm + 1; i < ne; i++)
                    if (prec(C->f, e[i], best)) best = e[i];
                C->sel_max[q] = best;
            }
        }
    }
    free(end_dn);
    free(end_up);
    return 0;
}

static void free_events(ctx_t *C)
{
    free(C->so); free(C->ev_ext); free(C->ev_nmin); free(C->ev_nmax); free(C->sel_min); free(C->sel_max);
    C->so = NULL; C->ev_ext = NULL; C->ev_nmin = C->ev_nmax = NULL; C->sel_min = C->sel_max = NULL;
}

int oracle_requests(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz,
                    uint8_t *req_out, int64_t *count_out);

static int correct_impl(const float *f, const float *fhat, int64_t nx, int64_t ny, int64_t nz,
                        float xi, int N, int64_t max_iters, int worklist, int events, int inc,
                        float *g, uint8_t *k, int64_t *info)
{
    /* info: [0] iterations, [1] residual, [2] status, [3] n_edits, [4] n_lossless */
    if (!dims_ok(nx, ny, nz) || !(xi > 0.0f) || !isfinite(xi) || N < 1 || N > 254 || max_iters < 0)
        return OR_EINVAL;
    derive_mesh();
    int64_t n = nx * ny * nz;
    for (int64_t p = 0; p < n; p++)
        if (!isfinite(f[p]) || !isfinite(fhat[p])) return OR_ENONFINITE;
    for (int64_t p = 0; p < n; p++) {
        float lo = f[p] - xi, hi = f[p] + xi;
        if (fhat[p] < lo || fhat[p] > hi) return OR_EBOUND;
    }
    ctx_t C;
    C.G.nx = nx; C.G.ny = ny; C.G.nz = nz; C.G.n = n;
    C.f = f;
    C.upf = malloc(sizeof(int64_t) * n);
    C.dnf = malloc(sizeof(int64_t) * n);
    C.tyf = malloc(n);
    C.o = malloc(sizeof(int64_t) * n);
    C.rank = malloc(sizeof(int64_t) * n);
    uint8_t *req = malloc(n), *active = malloc(n), *pact = malloc(n), *changed = malloc(n);
    if (!C.upf || !C.dnf || !C.tyf || !C.o || !C.rank || !req || !active || !pact || !changed) {
        free(C.upf); free(C.dnf); free(C.tyf); free(C.o); free(C.rank);
        free(req); free(active); free(pact); free(changed);
        return OR_ENOMEM;
    }
    oracle_classify(f, nx, ny, nz, C.upf, C.dnf, C.tyf);
    C.ncp = cp_order(f, C.tyf, n, C.o);
    for (int64_t p = 0; p < n; p++) C.rank[p] = -1;
    for (int64_t q = 0; q < C.ncp; q++) C.rank[C.o[q]] = q;
    C.events = events;
    C.inc = inc;
    C.so = NULL; C.ev_ext = NULL; C.ev_nmin = C.ev_nmax = NULL; C.sel_min = C.sel_max = NULL;
    if (events) {
        worklist = 0;  /* the event rules are evaluated in full every pass */
        if (setup_events(&C) != 0) {
            free_events(&C);
            free(C.upf); free(C.dnf); free(C.tyf); free(C.o); free(C.rank);
            free(req); free(active); free(pact); free(changed);
            return OR_ENOMEM;
        }
    }

    const float delta = xi / (float)N;
    for (int64_t p = 0; p < n; p++) {
        g[p] = fhat[p];
        k[p] = 0;
    }
    int64_t it = 0, residual = 0;
    int status = 0;
    int first = 1;
    for (;;) {
        int64_t nR;
        if (!worklist || first) {
            nR = check_full(&C, g, req);
        } else {
            /* Worklist: checkers in the closed neighbourhoods of the vertices
             * edited in the previous pass, pairs touching edited critical points. */
            memset(req, 0, (size_t)n);
            memset(active, 0, (size_t)n);
            memset(pact, 0, (size_t)n);
            for (int64_t x = 0; x < n; x++) {
                if (!changed[x]) continue;
                int64_t nb[32];
                int slot[32];
                int cnt = neighbours(&C.G, x, nb, slot);
                active[x] = 1;
                for (int j = 0; j < cnt; j++) active[nb[j]] = 1;
                int64_t r = C.rank[x];
                if (r >= 0) {
                    if (r >= 1) pact[r - 1] = 1;
                    if (r + 1 < C.ncp) pact[r] = 1;
                }
            }
#pragma omp parallel for schedule(dynamic, 4096)
            for (int64_t p = 0; p < n; p++)
                if (active[p]) check_vertex(&C, g, p, req);
            for (int64_t q = 0; q + 1 < C.ncp; q++)
                if (pact[q]) check_pair(&C, g, q, req);
            nR = -1; /* not the full |R| */
        }
        first = 0;
        int64_t nstar = 0;
        for (int64_t x = 0; x < n; x++)
            if (req[x] && k[x] <= N) nstar++;
        if (nstar == 0 || it == max_iters) {
            if (nR < 0) nR = check_full(&C, g, req);
            residual = nR;
            status = nstar != 0 ? OR_ITER_LIMIT : (nR == 0 ? OR_CONVERGED : OR_STUCK);
            break;
        }
        /* ApplyBoundedEdits: each requested, unpinned vertex once (decrements
         * of Delta down to fl(f - xi); increasing: increments up to fl(f + xi)). */
        for (int64_t x = 0; x < n; x++) {
            changed[x] = 0;
            if (!req[x] || k[x] > N) continue;
            float floor_x = inc ? f[x] + xi : f[x] - xi;
            if (k[x] < N) {
                float t = inc ? g[x] + delta : g[x] - delta;
                if (inc ? (t > floor_x) : (t < floor_x)) {
                    g[x] = floor_x;
                    k[x] = (uint8_t)(N + 1);
                } else {
                    g[x] = t;
                    k[x] = (uint8_t)(k[x] + 1);
                }
            } else {
                g[x] = floor_x;
                k[x] = (uint8_t)(N + 1);
            }
            changed[x] = 1;
        }
        it++;
    }
    int64_t ne = 0, nl = 0;
    for (int64_t p = 0; p < n; p++) {
        ne += k[p] > 0;
        nl += k[p] == N + 1;
    }
    info[0] = it;
    info[1] = residual;
    info[2] = status;
    info[3] = ne;
    info[4] = nl;
    free_events(&C);
    free(C.upf); free(C.dnf); free(C.tyf); free(C.o); free(C.rank);
    free(req); free(active); free(pact); free(changed);
    return 0;
}

/* Algorithm 1 with the EG constraints and the reformulated event constraints. */
int oracle_correct(const float *f, const float *fhat, int64_t nx, int64_t ny, int64_t nz,
                   float xi, int N, int64_t max_iters, int worklist,
                   float *g, uint8_t *k, int64_t *info)
{
    return correct_impl(f, fhat, nx, ny, nz, xi, N, max_iters, worklist, 0, 0, g, k, info);
}

/* Algorithm 1 with the EG constraints, the saddle-ordering constraints and the
 * original merge / split event constraints (C2, C3). */
int oracle_correct_events(const float *f, const float *fhat, int64_t nx, int64_t ny, int64_t nz,
                          float xi, int N, int64_t max_iters,
                          float *g, uint8_t *k, int64_t *info)
{
    return correct_impl(f, fhat, nx, ny, nz, xi, N, max_iters, 0, 1, 0, g, k, info);
}

/* Either constraint set (events) and either edit direction (increasing = 1:
 * every rule raises the vertex that must be higher, edits add Delta up to the
 * lossless bound fl(f + xi)). */
int oracle_correct_ex(const float *f, const float *fhat, int64_t nx, int64_t ny, int64_t nz,
                      float xi, int N, int64_t max_iters, int worklist, int events, int increasing,
                      float *g, uint8_t *k, int64_t *info)
{
    return correct_impl(f, fhat, nx, ny, nz, xi, N, max_iters, worklist, events, increasing != 0, g, k, info);
}

static int requests_impl(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz, int events, int inc,
                         uint8_t *req_out, int64_t *count_out);

/* The full request set R for a given edited field g (no pinned filter). */
int oracle_requests(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz,
                    uint8_t *req_out, int64_t *count_out)
{
    return requests_impl(f, g, nx, ny, nz, 0, 0, req_out, count_out);
}

/* The same with the original event constraints in place of R3. */
int oracle_requests_events(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz,
                           uint8_t *req_out, int64_t *count_out)
{
    return requests_impl(f, g, nx, ny, nz, 1, 0, req_out, count_out);
}

/* Either constraint set and either edit direction. */
int oracle_requests_ex(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz, int events,
                       int increasing, uint8_t *req_out, int64_t *count_out)
{
    return requests_impl(f, g, nx, ny, nz, events, increasing != 0, req_out, count_out);
}

static int requests_impl(const float *f, const float *g, int64_t nx, int64_t ny, int64_t nz, int events, int inc,
                         uint8_t *req_out, int64_t *count_out)
{
    if (!dims_ok(nx, ny, nz)) return OR_EINVAL;
    derive_mesh();
    int64_t n = nx * ny * nz;
    ctx_t C;
    C.G.nx = nx; C.G.ny = ny; C.G.nz = nz; C.G.n = n;
    C.f = f;
    C.upf = malloc(sizeof(int64_t) * n);
    C.dnf = malloc(sizeof(int64_t) * n);
    C.tyf = malloc(n);
    C.o = malloc(sizeof(int64_t) * n);
    C.rank = NULL;
    if (!C.upf || !C.dnf || !C.tyf || !C.o) {
        free(C.upf); free(C.dnf); free(C.tyf); free(C.o);
        return OR_ENOMEM;
    }
    oracle_classify(f, nx, ny, nz, C.upf, C.dnf, C.tyf);
    C.ncp = cp_order(f, C.tyf, n, C.o);
    C.events = events;
    C.inc = inc;
    C.so = NULL; C.ev_ext = NULL; C.ev_nmin = C.ev_nmax = NULL; C.sel_min = C.sel_max = NULL;
    if (events && setup_events(&C) != 0) {
        free_events(&C);
        free(C.upf); free(C.dnf); free(C.tyf); free(C.o);
        return OR_ENOMEM;
    }
    *count_out = check_full(&C, g, req_out);
    free_events(&C);
    free(C.upf); free(C.dnf); free(C.tyf); free(C.o);
    return 0;
}
