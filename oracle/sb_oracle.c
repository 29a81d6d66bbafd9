/*
 * sb_oracle.c -- plain, slow CPU oracle for the parallel sparse-blossom decoder.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference leg use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper: "Decoding task" paragraph; SI Sec. S1 "Preliminaries
 * on sparse blossom"; Methods, Algorithms 1 and 2):
 *
 *  1. The detector graph with parallel edges merged (minimum weight, ties to the
 *     lower input index), internal weights 2w so every event lies at an integer
 *     time (SI S1, last paragraph before the event list).
 *  2. Exact graph distances by Dijkstra from every detection event; graph-fill
 *     regions are the balls of radius Rad(s) around each event s in this metric,
 *     where Rad(s) is the sum of the dual values of s and of every blossom
 *     containing s (SI S1: a blossom updates only its own dual, the area of a
 *     blossom is its children's area grown by the blossom dual).
 *  3. The sparse-blossom event loop (SI S1, events (a)-(g)) with one uniform
 *     dual step for every tree (delta = 1 per unit time): at each step the due
 *     event with the smallest canonical key (t, kind, lo, hi) is applied, where
 *     kind orders IMPLODE < COLLIDE < BOUNDARY and lo < hi are detection-event
 *     ranks (position in the sorted event list).  Due events are found by brute
 *     force over every pair of events.
 *  4. Output: expand blossoms into a perfect embedded matching, report its
 *     weight (original units) and the XOR of the observable masks of canonical
 *     shortest paths (Dijkstra tree of the lower-ranked endpoint, predecessor =
 *     lowest edge id among tight edges; to the boundary: lowest boundary edge id
 *     among the minimal ones).
 *  5. Hierarchical mode: Algorithm 1 (processing clusters from the detection
 *     events with the (d_k, b_k) of Algorithm 3) and the hierarchical execution
 *     rule of Algorithm 2, simulated sequentially like the paper's simulator
 *     (Methods, "Numerical evaluation"): each cluster runs from t = 0 with every
 *     retained lower-level configuration present as frozen regions.
 *  6. Parallel event count E_ideal (Methods, "Numerical evaluation"): per
 *     cluster, its stopping time and the times of its events; the critical
 *     path through the levels combines them level by level (the recursion is
 *     written out where the levels run).  An event is one step of the loop of
 *     item 3 (an implosion, a collision or a boundary contact); global mode
 *     reports its whole event count.
 *
 * Checks computed for the tests: primal objective == dual objective (sum of all
 * duals equals the matched weight in internal units), dual feasibility of every
 * pair and boundary constraint, and the unique-touching rule of Alg. 2.
 */
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_INF (LLONG_MAX / 8)
#define BND_KEY INT_MAX

enum { ST_OK = 0, ST_NO_SOLUTION = 1, ST_BUDGET = 2, ST_INTERNAL = 3, ST_BADARG = 4 };
enum { K_IMPLODE = 0, K_COLLIDE = 1, K_BOUNDARY = 2 };
enum { MATE_NONE = -1, MATE_BOUNDARY = -2 };

/* ------------------------------------------------------------------------- */
/* Graph                                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n, m;
    int *eu, *ev;          /* ev == -1: boundary edge */
    long long *ew;         /* internal weight = 2 * original weight */
    uint64_t *eobs;
    int *adj_off, *adj_e;  /* incident merged edges of each detector */
    long long wmax;        /* largest internal weight */
} OGraph;

typedef struct {
    int lo, hi, w, idx;
} PhysKey;

static int cmp_phys(const void *a, const void *b) {
    const PhysKey *x = (const PhysKey *)a, *y = (const PhysKey *)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

void or_graph_free(OGraph *g) {
    if (!g) return;
    free(g->eu); free(g->ev); free(g->ew); free(g->eobs);
    free(g->adj_off); free(g->adj_e);
    free(g);
}

/* Merge physical edges: one merged edge per (lo, hi) detector pair or per
 * (detector, boundary); it keeps the smallest weight, ties to the lower input
 * index, and that edge's observable mask.  Merged edge ids follow (lo, hi)
 * order with the boundary sorting after every detector partner. */
int or_graph_build(int n, int m, const int *u, const int *v, const int *w,
                   const uint64_t *obs, OGraph **out) {
    *out = NULL;
    if (n <= 0 || m < 0) return ST_BADARG;
    PhysKey *k = (PhysKey *)malloc(sizeof(PhysKey) * (size_t)(m > 0 ? m : 1));
    for (int i = 0; i < m; i++) {
        if (u[i] < 0 || u[i] >= n || v[i] < -1 || v[i] >= n || u[i] == v[i] || w[i] <= 0) {
            free(k);
            return ST_BADARG;
        }
        if (v[i] < 0) { k[i].lo = u[i]; k[i].hi = BND_KEY; }
        else { k[i].lo = u[i] < v[i] ? u[i] : v[i]; k[i].hi = u[i] < v[i] ? v[i] : u[i]; }
        k[i].w = w[i];
        k[i].idx = i;
    }
    qsort(k, (size_t)m, sizeof(PhysKey), cmp_phys);
    OGraph *g = (OGraph *)calloc(1, sizeof(OGraph));
    g->n = n;
    g->eu = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    g->ev = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    g->ew = (long long *)malloc(sizeof(long long) * (size_t)(m + 1));
    g->eobs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m + 1));
    int mm = 0;
    for (int i = 0; i < m; i++) {
        if (i > 0 && k[i].lo == k[i - 1].lo && k[i].hi == k[i - 1].hi) continue;
        g->eu[mm] = k[i].lo;
        g->ev[mm] = k[i].hi == BND_KEY ? -1 : k[i].hi;
        g->ew[mm] = 2LL * k[i].w;
        g->eobs[mm] = obs[k[i].idx];
        mm++;
    }
    free(k);
    g->m = mm;
    g->wmax = 0;
    for (int e = 0; e < mm; e++)
        if (g->ew[e] > g->wmax) g->wmax = g->ew[e];
    g->adj_off = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int e = 0; e < mm; e++) {
        g->adj_off[g->eu[e] + 1]++;
        if (g->ev[e] >= 0) g->adj_off[g->ev[e] + 1]++;
    }
    for (int x = 0; x < n; x++) g->adj_off[x + 1] += g->adj_off[x];
    g->adj_e = (int *)malloc(sizeof(int) * (size_t)(g->adj_off[n] + 1));
    int *fill = (int *)calloc((size_t)n, sizeof(int));
    for (int e = 0; e < mm; e++) {
        int a = g->eu[e], b = g->ev[e];
        g->adj_e[g->adj_off[a] + fill[a]++] = e;
        if (b >= 0) g->adj_e[g->adj_off[b] + fill[b]++] = e;
    }
    free(fill);
    *out = g;
    return ST_OK;
}

int or_graph_num_edges(const OGraph *g) { return g->m; }
long long or_graph_wmax(const OGraph *g) { return g->wmax; }

void or_graph_edges(const OGraph *g, int *u, int *v, long long *w, uint64_t *obs) {
    for (int e = 0; e < g->m; e++) {
        u[e] = g->eu[e]; v[e] = g->ev[e]; w[e] = g->ew[e]; obs[e] = g->eobs[e];
    }
}

/* ------------------------------------------------------------------------- */
/* Dijkstra with canonical predecessors                                       */
/* ------------------------------------------------------------------------- */

typedef struct { long long d; int x; } HeapItem;

static void heap_push(HeapItem *h, int *sz, HeapItem it) {
    int i = (*sz)++;
    h[i] = it;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        HeapItem t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static HeapItem heap_pop(HeapItem *h, int *sz) {
    HeapItem top = h[0];
    h[0] = h[--(*sz)];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, s = i;
        if (l < *sz && h[l].d < h[s].d) s = l;
        if (r < *sz && h[r].d < h[s].d) s = r;
        if (s == i) break;
        HeapItem t = h[s]; h[s] = h[i]; h[i] = t;
        i = s;
    }
    return top;
}

/* dist[x] = shortest internal-weight distance from src (OR_INF if unreachable);
 * pred[x] = lowest edge id e = (y, x) with dist[y] + w(e) == dist[x], -1 at src. */
static void dijkstra(const OGraph *g, int src, long long *dist, int *pred) {
    int n = g->n;
    for (int x = 0; x < n; x++) { dist[x] = OR_INF; pred[x] = -1; }
    HeapItem *h = (HeapItem *)malloc(sizeof(HeapItem) * (size_t)(2 * g->m + n + 4));
    int sz = 0;
    dist[src] = 0;
    heap_push(h, &sz, (HeapItem){0, src});
    while (sz > 0) {
        HeapItem it = heap_pop(h, &sz);
        if (it.d != dist[it.x]) continue;
        for (int j = g->adj_off[it.x]; j < g->adj_off[it.x + 1]; j++) {
            int e = g->adj_e[j];
            int y = g->eu[e] == it.x ? g->ev[e] : g->eu[e];
            if (y < 0) continue;
            long long nd = it.d + g->ew[e];
            if (nd < dist[y]) { dist[y] = nd; heap_push(h, &sz, (HeapItem){nd, y}); }
        }
    }
    free(h);
    for (int e = 0; e < g->m; e++) {
        int a = g->eu[e], b = g->ev[e];
        if (b < 0) continue;
        if (dist[a] < OR_INF && dist[a] + g->ew[e] == dist[b] && pred[b] < 0 && b != src) pred[b] = e;
        if (dist[b] < OR_INF && dist[b] + g->ew[e] == dist[a] && pred[a] < 0 && a != src) pred[a] = e;
    }
}

static uint64_t path_obs(const OGraph *g, const int *pred, int src, int x) {
    uint64_t o = 0;
    while (x != src) {
        int e = pred[x];
        o ^= g->eobs[e];
        x = g->eu[e] == x ? g->ev[e] : g->eu[e];
    }
    return o;
}

/* Per-shot geometry: pair distances, boundary distances and path observables. */
typedef struct {
    int k;
    int *det;              /* sorted detection events */
    long long *D;          /* k*k */
    uint64_t *PO;          /* k*k canonical pair-path observables */
    long long *BD;         /* k, OR_INF if no boundary reachable */
    int *BE;               /* k, canonical boundary edge id or -1 */
    uint64_t *BO;          /* k */
} Geo;

static void geo_free(Geo *q) {
    free(q->det); free(q->D); free(q->PO); free(q->BD); free(q->BE); free(q->BO);
}

static void geo_build(const OGraph *g, int k, const int *det, Geo *q) {
    q->k = k;
    q->det = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    memcpy(q->det, det, sizeof(int) * (size_t)k);
    q->D = (long long *)malloc(sizeof(long long) * (size_t)(k * k + 1));
    q->PO = (uint64_t *)calloc((size_t)(k * k + 1), sizeof(uint64_t));
    q->BD = (long long *)malloc(sizeof(long long) * (size_t)(k + 1));
    q->BE = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    q->BO = (uint64_t *)calloc((size_t)(k + 1), sizeof(uint64_t));
    long long *dist = (long long *)malloc(sizeof(long long) * (size_t)g->n);
    int *pred = (int *)malloc(sizeof(int) * (size_t)g->n);
    for (int a = 0; a < k; a++) {
        dijkstra(g, det[a], dist, pred);
        for (int b = 0; b < k; b++) {
            q->D[a * k + b] = dist[det[b]];
            if (b > a && dist[det[b]] < OR_INF) {
                uint64_t o = path_obs(g, pred, det[a], det[b]);
                q->PO[a * k + b] = o;
                q->PO[b * k + a] = o;
            }
        }
        long long bd = OR_INF;
        int be = -1;
        for (int e = 0; e < g->m; e++) {
            if (g->ev[e] >= 0 || dist[g->eu[e]] >= OR_INF) continue;
            long long c = dist[g->eu[e]] + g->ew[e];
            if (c < bd) { bd = c; be = e; }
        }
        q->BD[a] = bd;
        q->BE[a] = be;
        q->BO[a] = be >= 0 ? (g->eobs[be] ^ path_obs(g, pred, det[a], g->eu[be])) : 0;
    }
    free(dist); free(pred);
}

/* ------------------------------------------------------------------------- */
/* Matcher: sparse-blossom dynamics on graph-fill regions (SI S1)             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int k, cap, nnodes;
    const Geo *q;
    long long t;
    int *present;                 /* leaf takes part in the current run */
    long long *y;
    int *alive, *bpar, *label;
    int *tpar, *tps, *tpo;        /* tree parent, leaf on own side, leaf on parent side */
    int *mate, *ms, *mo;          /* mate node / MATE_*, own leaf, partner leaf (-1 boundary) */
    int *clen;                    /* blossom cycle length (0 for leaves) */
    int **cnode, **cs, **co;      /* edge i joins cnode[i] (leaf cs[i]) and cnode[i+1] (leaf co[i]) */
    int *config;                  /* retained-configuration id of each node */
    int *touched;
    long long events[3];
    long long *evt;               /* time of every applied event, in order */
    long long nev, evcap;
    long long budget;
    int status;
} Matcher;

static void m_init(Matcher *M, const Geo *q) {
    int k = q->k;
    memset(M, 0, sizeof(*M));
    M->k = k;
    M->q = q;
    M->cap = 4 * k + 8;
    int c = M->cap;
    M->present = (int *)calloc((size_t)k + 1, sizeof(int));
    M->y = (long long *)calloc((size_t)c, sizeof(long long));
    M->alive = (int *)calloc((size_t)c, sizeof(int));
    M->bpar = (int *)malloc(sizeof(int) * (size_t)c);
    M->label = (int *)calloc((size_t)c, sizeof(int));
    M->tpar = (int *)malloc(sizeof(int) * (size_t)c);
    M->tps = (int *)malloc(sizeof(int) * (size_t)c);
    M->tpo = (int *)malloc(sizeof(int) * (size_t)c);
    M->mate = (int *)malloc(sizeof(int) * (size_t)c);
    M->ms = (int *)malloc(sizeof(int) * (size_t)c);
    M->mo = (int *)malloc(sizeof(int) * (size_t)c);
    M->clen = (int *)calloc((size_t)c, sizeof(int));
    M->cnode = (int **)calloc((size_t)c, sizeof(int *));
    M->cs = (int **)calloc((size_t)c, sizeof(int *));
    M->co = (int **)calloc((size_t)c, sizeof(int *));
    M->config = (int *)malloc(sizeof(int) * (size_t)c);
    M->touched = (int *)calloc((size_t)c, sizeof(int));
    for (int i = 0; i < c; i++) {
        M->bpar[i] = -1; M->tpar[i] = -1; M->tps[i] = M->tpo[i] = -1;
        M->mate[i] = MATE_NONE; M->ms[i] = M->mo[i] = -1; M->config[i] = -1;
    }
    M->nnodes = k;
    M->budget = 50000000LL;
}

static void m_free(Matcher *M) {
    for (int i = 0; i < M->cap; i++) { free(M->cnode[i]); free(M->cs[i]); free(M->co[i]); }
    free(M->present); free(M->y); free(M->alive); free(M->bpar); free(M->label);
    free(M->tpar); free(M->tps); free(M->tpo); free(M->mate); free(M->ms); free(M->mo);
    free(M->clen); free(M->cnode); free(M->cs); free(M->co); free(M->config); free(M->touched);
    free(M->evt);
}

static void m_log_event(Matcher *M, long long t) {
    if (M->nev == M->evcap) {
        M->evcap = M->evcap ? 2 * M->evcap : 64;
        M->evt = (long long *)realloc(M->evt, sizeof(long long) * (size_t)M->evcap);
    }
    M->evt[M->nev++] = t;
}

/* A leaf joins the run as a fresh root: radius 0, growing. */
static void m_add_root(Matcher *M, int a) {
    M->present[a] = 1;
    M->alive[a] = 1;
    M->y[a] = 0;
    M->bpar[a] = -1;
    M->label[a] = +1;
    M->tpar[a] = -1;
    M->mate[a] = MATE_NONE;
}

static int m_top(const Matcher *M, int v) {
    while (M->bpar[v] >= 0) v = M->bpar[v];
    return v;
}

static long long m_rad(const Matcher *M, int a) {
    long long r = 0;
    for (int v = a; v >= 0; v = M->bpar[v]) r += M->y[v];
    return r;
}

static int m_root(const Matcher *M, int v) {
    while (M->tpar[v] >= 0) v = M->tpar[v];
    return v;
}

static int m_contains(const Matcher *M, int node, int leaf) {
    for (int v = leaf; v >= 0; v = M->bpar[v])
        if (v == node) return 1;
    return 0;
}

static int m_min_leaf(const Matcher *M, int node) {
    for (int a = 0; a < M->k; a++)
        if (M->present[a] && m_contains(M, node, a)) return a;
    return -1;
}

/* Child of blossom b that contains leaf a. */
static int m_child_index(const Matcher *M, int b, int a) {
    int v = a;
    while (M->bpar[v] != b) v = M->bpar[v];
    for (int i = 0; i < M->clen[b]; i++)
        if (M->cnode[b][i] == v) return i;
    return -1;
}

static void m_touch(Matcher *M, int v) { M->touched[v] = 1; }

static int m_new_node(Matcher *M) {
    for (int i = M->k; i < M->cap; i++)
        if (!M->alive[i] && M->clen[i] == 0 && M->cnode[i] == NULL) {
            if (i >= M->nnodes) M->nnodes = i + 1;
            return i;
        }
    return -1;
}

/* Top-level nodes whose tree root is r. */
static int m_tree_members(const Matcher *M, int r, int *out) {
    int c = 0;
    for (int v = 0; v < M->nnodes; v++)
        if (M->alive[v] && M->bpar[v] < 0 && M->label[v] != 0 && m_root(M, v) == r) out[c++] = v;
    return c;
}

/* Flip matches along the tree path from outer node A to its root. */
static void m_augment_to_root(Matcher *M, int A) {
    int v = A;
    while (M->tpar[v] >= 0) {
        int I = M->tpar[v];
        int O = M->tpar[I];
        M->mate[I] = O; M->ms[I] = M->tps[I]; M->mo[I] = M->tpo[I];
        M->mate[O] = I; M->ms[O] = M->tpo[I]; M->mo[O] = M->tps[I];
        v = O;
    }
}

static void m_freeze(Matcher *M, const int *mem, int c) {
    for (int i = 0; i < c; i++) {
        M->label[mem[i]] = 0;
        M->tpar[mem[i]] = -1;
        M->tps[mem[i]] = M->tpo[mem[i]] = -1;
    }
}

/* Events (b), (f), (g): augment the tree(s) and freeze them. */
static void m_augment(Matcher *M, int A, int a, int B, int b) {
    int *mem = (int *)malloc(sizeof(int) * (size_t)(2 * M->nnodes + 2));
    int c = m_tree_members(M, m_root(M, A), mem);
    if (B >= 0 && M->label[B] == +1) c += m_tree_members(M, m_root(M, B), mem + c);
    for (int i = 0; i < c; i++) m_touch(M, mem[i]);
    m_augment_to_root(M, A);
    if (B >= 0 && M->label[B] == +1) m_augment_to_root(M, B);
    if (B >= 0) {
        M->mate[A] = B; M->ms[A] = a; M->mo[A] = b;
        M->mate[B] = A; M->ms[B] = b; M->mo[B] = a;
        m_touch(M, B);
    } else {
        M->mate[A] = MATE_BOUNDARY; M->ms[A] = a; M->mo[A] = -1;
    }
    m_freeze(M, mem, c);
    free(mem);
}

/* Event (a): outer A touches frozen B (matched to C): B inner, C outer. */
static void m_grow(Matcher *M, int A, int a, int B, int b) {
    int C = M->mate[B];
    M->label[B] = -1;
    M->tpar[B] = A; M->tps[B] = b; M->tpo[B] = a;
    M->label[C] = +1;
    M->tpar[C] = B; M->tps[C] = M->ms[C]; M->tpo[C] = M->mo[C];
    m_touch(M, B); m_touch(M, C); m_touch(M, A);
}

/* Event (c): outer A and outer B of one tree collide -> new blossom. */
static int m_blossom(Matcher *M, int A, int a, int B, int b) {
    int cap = M->nnodes + 2;
    int *pa = (int *)malloc(sizeof(int) * (size_t)cap);
    int *pb = (int *)malloc(sizeof(int) * (size_t)cap);
    int na = 0, nb = 0;
    for (int v = A; v >= 0; v = M->tpar[v]) pa[na++] = v;
    for (int v = B; v >= 0; v = M->tpar[v]) pb[nb++] = v;
    /* strip the common suffix (ancestors above the lowest common ancestor) */
    while (na > 1 && nb > 1 && pa[na - 2] == pb[nb - 2]) { na--; nb--; }
    int L = pa[na - 1];
    if (L != pb[nb - 1]) { free(pa); free(pb); return ST_INTERNAL; }
    int m = na + nb - 1;
    int N = m_new_node(M);
    if (N < 0) { free(pa); free(pb); return ST_INTERNAL; }
    int *cn = (int *)malloc(sizeof(int) * (size_t)m);
    int *cs = (int *)malloc(sizeof(int) * (size_t)m);
    int *co = (int *)malloc(sizeof(int) * (size_t)m);
    int i = 0;
    /* LCA, then down the A side (pa reversed, without the LCA) */
    cn[i++] = L;
    for (int j = na - 2; j >= 0; j--) cn[i++] = pa[j];
    /* then the B side going up (pb without the LCA) */
    for (int j = 0; j <= nb - 2; j++) cn[i++] = pb[j];
    int ia = na - 1; /* index of A in the cycle (0 when A is the LCA) */
    for (int j = 0; j < m; j++) {
        int x = cn[j], z = cn[(j + 1) % m];
        if (j < ia) {            /* z is the tree child of x */
            cs[j] = M->tpo[z]; co[j] = M->tps[z];
        } else if (j == ia) {    /* the colliding pair */
            cs[j] = a; co[j] = b;
        } else {                 /* x is the tree child of z */
            cs[j] = M->tps[x]; co[j] = M->tpo[x];
        }
    }
    M->alive[N] = 1;
    M->y[N] = 0;
    M->bpar[N] = -1;
    M->label[N] = +1;
    M->tpar[N] = M->tpar[L]; M->tps[N] = M->tps[L]; M->tpo[N] = M->tpo[L];
    M->mate[N] = M->mate[L]; M->ms[N] = M->ms[L]; M->mo[N] = M->mo[L];
    M->clen[N] = m; M->cnode[N] = cn; M->cs[N] = cs; M->co[N] = co;
    M->config[N] = M->config[L];
    M->touched[N] = 1;
    for (int j = 0; j < m; j++) { M->bpar[cn[j]] = N; m_touch(M, cn[j]); }
    for (int v = 0; v < M->nnodes; v++) {
        if (!M->alive[v] || M->bpar[v] >= 0 || v == N) continue;
        if (M->tpar[v] >= 0 && M->bpar[M->tpar[v]] == N) M->tpar[v] = N;
        if (M->mate[v] >= 0 && M->bpar[M->mate[v]] == N) M->mate[v] = N;
    }
    free(pa); free(pb);
    return ST_OK;
}

/* Event (d): inner blossom B with zero dual shatters (SI S1, EXPAND). */
static int m_shatter(Matcher *M, int B) {
    int m = M->clen[B];
    int *cn = M->cnode[B], *cs = M->cs[B], *co = M->co[B];
    int P = M->tpar[B], C = M->mate[B];
    int ip = m_child_index(M, B, M->tps[B]);
    int ic = m_child_index(M, B, M->ms[B]);
    if (ip < 0 || ic < 0 || C < 0) return ST_INTERNAL;
    int fwd = ((ic - ip) % m + m) % m;
    int dir = (fwd % 2 == 0) ? +1 : -1;
    int L = dir > 0 ? fwd : m - fwd;
    for (int j = 0; j < m; j++) { M->bpar[cn[j]] = -1; m_touch(M, cn[j]); }
    /* path q_0 .. q_L from the child holding the parent edge to the one holding the mate */
    int prev = -1;
    for (int j = 0; j <= L; j++) {
        int idx = ((ip + dir * j) % m + m) % m;
        int q = cn[idx];
        M->label[q] = (j % 2 == 0) ? -1 : +1;
        if (j == 0) {
            M->tpar[q] = P; M->tps[q] = M->tps[B]; M->tpo[q] = M->tpo[B];
        } else {
            int pidx = ((ip + dir * (j - 1)) % m + m) % m;
            int self, other; /* leaf in q, leaf in prev */
            if (dir > 0) { self = co[pidx]; other = cs[pidx]; }
            else { self = cs[idx]; other = co[idx]; }
            M->tpar[q] = prev; M->tps[q] = self; M->tpo[q] = other;
            if (j % 2 == 1) { /* outer q is matched to its inner parent */
                M->mate[q] = prev; M->ms[q] = self; M->mo[q] = other;
                M->mate[prev] = q; M->ms[prev] = other; M->mo[prev] = self;
            }
        }
        prev = q;
    }
    int qL = prev;
    M->mate[qL] = C; M->ms[qL] = M->ms[B]; M->mo[qL] = M->mo[B];
    M->mate[C] = qL;
    M->tpar[C] = qL;
    /* remaining children, in pairs along the cycle, frozen */
    int rem = m - 1 - L;
    for (int j = 1; j <= rem; j += 2) {
        int i1 = ((ic + dir * j) % m + m) % m;
        int i2 = ((ic + dir * (j + 1)) % m + m) % m;
        int x = cn[i1], z = cn[i2];
        int lx, lz;
        if (dir > 0) { lx = cs[i1]; lz = co[i1]; }
        else { lx = co[i2]; lz = cs[i2]; }
        M->label[x] = 0; M->label[z] = 0;
        M->tpar[x] = M->tpar[z] = -1;
        M->mate[x] = z; M->ms[x] = lx; M->mo[x] = lz;
        M->mate[z] = x; M->ms[z] = lz; M->mo[z] = lx;
    }
    if (P >= 0) { /* nothing points at B except P's child link (tpar of B) and C */ }
    M->alive[B] = 0;
    free(M->cnode[B]); free(M->cs[B]); free(M->co[B]);
    M->cnode[B] = M->cs[B] = M->co[B] = NULL;
    M->clen[B] = 0;
    M->tpar[B] = -1; M->mate[B] = MATE_NONE; M->bpar[B] = -1; M->y[B] = 0;
    return ST_OK;
}

typedef struct { long long t; int kind, lo, hi; } Ev;

static int ev_less(const Ev *x, const Ev *y) {
    if (x->t != y->t) return x->t < y->t;
    if (x->kind != y->kind) return x->kind < y->kind;
    if (x->lo != y->lo) return x->lo < y->lo;
    return x->hi < y->hi;
}

/* Run the event loop until no growing region is left. */
static int m_run(Matcher *M) {
    const Geo *q = M->q;
    int k = M->k;
    long long *rad = (long long *)malloc(sizeof(long long) * (size_t)(k + 1));
    int *top = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    for (long long iter = 0;; iter++) {
        if (iter > M->budget) { free(rad); free(top); return ST_BUDGET; }
        for (int a = 0; a < k; a++) {
            if (!M->present[a]) continue;
            top[a] = m_top(M, a);
            rad[a] = m_rad(M, a);
        }
        int any_outer = 0;
        Ev best = {OR_INF, 9, INT_MAX, INT_MAX};
        int have = 0;
        for (int a = 0; a < k; a++) {
            if (!M->present[a]) continue;
            int A = top[a];
            if (M->label[A] == +1) any_outer = 1;
            for (int b = a + 1; b < k; b++) {
                if (!M->present[b]) continue;
                int B = top[b];
                if (A == B) continue;
                int r = M->label[A] + M->label[B];
                if (r <= 0) continue;
                long long dab = q->D[a * k + b];
                if (dab >= OR_INF) continue;
                long long gap = dab - rad[a] - rad[b];
                if (gap < 0 || gap % r != 0) { free(rad); free(top); return ST_INTERNAL; }
                Ev e = {M->t + gap / r, K_COLLIDE, a, b};
                if (!have || ev_less(&e, &best)) { best = e; have = 1; }
            }
            if (M->label[A] == +1 && q->BD[a] < OR_INF) {
                long long gap = q->BD[a] - rad[a];
                if (gap < 0) { free(rad); free(top); return ST_INTERNAL; }
                Ev e = {M->t + gap, K_BOUNDARY, a, INT_MAX};
                if (!have || ev_less(&e, &best)) { best = e; have = 1; }
            }
        }
        for (int v = k; v < M->nnodes; v++) {
            if (!M->alive[v] || M->bpar[v] >= 0 || M->label[v] != -1) continue;
            Ev e = {M->t + M->y[v], K_IMPLODE, m_min_leaf(M, v), 0};
            if (!have || ev_less(&e, &best)) { best = e; have = 1; }
        }
        if (!any_outer) break;
        if (!have) { free(rad); free(top); return ST_NO_SOLUTION; }
        /* an inner region never shrinks below zero */
        long long dt = best.t - M->t;
        for (int v = 0; v < M->nnodes; v++)
            if (M->alive[v] && M->bpar[v] < 0 && M->label[v] == -1 && M->y[v] < dt) {
                free(rad); free(top); return ST_INTERNAL;
            }
        for (int v = 0; v < M->nnodes; v++)
            if (M->alive[v] && M->bpar[v] < 0) M->y[v] += (long long)M->label[v] * dt;
        M->t = best.t;
        M->events[best.kind]++;
        m_log_event(M, best.t);
        int st = ST_OK;
        if (best.kind == K_IMPLODE) {
            int B = m_top(M, best.lo);
            st = m_shatter(M, B);
        } else if (best.kind == K_BOUNDARY) {
            int A = m_top(M, best.lo);
            m_augment(M, A, best.lo, -1, -1);
        } else {
            int a = best.lo, b = best.hi;
            int A = m_top(M, a), B = m_top(M, b);
            if (M->label[A] != +1) { int tt = A; A = B; B = tt; tt = a; a = b; b = tt; }
            if (M->label[B] == +1) {
                if (m_root(M, A) == m_root(M, B)) st = m_blossom(M, A, a, B, b);
                else m_augment(M, A, a, B, b);
            } else if (M->label[B] == 0) {
                if (M->mate[B] == MATE_BOUNDARY) m_augment(M, A, a, B, b);
                else if (M->mate[B] >= 0) m_grow(M, A, a, B, b);
                else st = ST_INTERNAL;
            } else {
                st = ST_INTERNAL;
            }
        }
        if (st != ST_OK) { free(rad); free(top); return st; }
    }
    free(rad); free(top);
    return ST_OK;
}

/* Expand blossom `node` whose externally matched leaf is `ext`; append the
 * internal leaf-level matched pairs. */
static void m_expand(const Matcher *M, int node, int ext, int *pa, int *pb, int *np) {
    if (node < M->k) return;
    int m = M->clen[node];
    int i0 = m_child_index(M, node, ext);
    m_expand(M, M->cnode[node][i0], ext, pa, pb, np);
    for (int j = 1; j < m; j += 2) {
        int i1 = (i0 + j) % m, i2 = (i0 + j + 1) % m;
        int x = M->cnode[node][i1], z = M->cnode[node][i2];
        int lx = M->cs[node][i1], lz = M->co[node][i1];
        pa[*np] = lx; pb[*np] = lz; (*np)++;
        m_expand(M, x, lx, pa, pb, np);
        m_expand(M, z, lz, pa, pb, np);
    }
}

typedef struct {
    long long weight;          /* original units */
    uint64_t obs;
    int status;
    long long events_implode, events_collide, events_boundary;
    long long dual_sum;        /* sum of every dual, internal units */
    long long primal_internal; /* matched weight, internal units */
    int dual_feasible;         /* every pair / boundary slack >= 0 */
    int tight;                 /* every matched edge has zero slack */
    int touch_violations;      /* Alg. 2 unique-touching breaches */
    int num_levels;            /* highest processing-cluster level (hierarchical) */
    int num_clusters;
    int level1_events;         /* detection events resolved at level 1 */
    long long stop_time;       /* largest stop time of any run */
    long long e_ideal;         /* parallel event count (Methods, "Numerical evaluation") */
    long long t_ideal;         /* its critical-path stopping time, internal units */
} OResult;

/* Mark the edges of the canonical path from detector src to detector x
 * (XOR into corr, one byte per merged edge). */
static void mark_path(const OGraph *g, int src, int x, unsigned char *corr) {
    long long *dist = (long long *)malloc(sizeof(long long) * (size_t)g->n);
    int *pred = (int *)malloc(sizeof(int) * (size_t)g->n);
    dijkstra(g, src, dist, pred);
    while (x != src) {
        int e = pred[x];
        corr[e] ^= 1;
        x = g->eu[e] == x ? g->ev[e] : g->eu[e];
    }
    free(dist); free(pred);
}

static void m_finish(Matcher *M, OResult *res, const OGraph *g, unsigned char *corr) {
    const Geo *q = M->q;
    int k = M->k;
    int *pa = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    int *pb = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    int np = 0, nbd = 0;
    int *bl = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    for (int v = 0; v < M->nnodes; v++) {
        if (!M->alive[v] || M->bpar[v] >= 0) continue;
        if (M->mate[v] == MATE_BOUNDARY) {
            bl[nbd++] = M->ms[v];
            m_expand(M, v, M->ms[v], pa, pb, &np);
        } else if (M->mate[v] >= 0 && v < M->mate[v]) {
            pa[np] = M->ms[v]; pb[np] = M->mo[v]; np++;
            m_expand(M, v, M->ms[v], pa, pb, &np);
            m_expand(M, M->mate[v], M->mo[v], pa, pb, &np);
        }
    }
    long long wi = 0;
    uint64_t ob = 0;
    int tight = 1;
    for (int i = 0; i < np; i++) {
        int a = pa[i], b = pb[i];
        wi += q->D[a * k + b];
        ob ^= q->PO[a * k + b];
    }
    for (int i = 0; i < nbd; i++) {
        wi += q->BD[bl[i]];
        ob ^= q->BO[bl[i]];
    }
    if (corr) {
        memset(corr, 0, (size_t)g->m);
        for (int i = 0; i < np; i++) {
            int a = pa[i] < pb[i] ? pa[i] : pb[i], b = pa[i] < pb[i] ? pb[i] : pa[i];
            mark_path(g, q->det[a], q->det[b], corr);
        }
        for (int i = 0; i < nbd; i++) {
            int e = q->BE[bl[i]];
            corr[e] ^= 1;
            mark_path(g, q->det[bl[i]], g->eu[e], corr);
        }
    }
    long long ds = 0;
    for (int v = 0; v < M->nnodes; v++)
        if (M->alive[v]) ds += M->y[v];
    /* dual feasibility: slack(a,b) = D - duals of regions holding exactly one of a, b */
    int feas = 1;
    for (int a = 0; a < k; a++) {
        if (!M->present[a]) continue;
        long long ra = m_rad(M, a);
        if (q->BD[a] < OR_INF && q->BD[a] - ra < 0) feas = 0;
        for (int b = a + 1; b < k; b++) {
            if (!M->present[b] || q->D[a * k + b] >= OR_INF) continue;
            long long s = q->D[a * k + b] - ra - m_rad(M, b);
            for (int v = M->bpar[a]; v >= 0; v = M->bpar[v])
                if (m_contains(M, v, b)) s += 2 * M->y[v];
            if (s < 0) feas = 0;
        }
    }
    for (int i = 0; i < np; i++) {
        int a = pa[i], b = pb[i];
        long long s = q->D[a * k + b] - m_rad(M, a) - m_rad(M, b);
        for (int v = M->bpar[a]; v >= 0; v = M->bpar[v])
            if (m_contains(M, v, b)) s += 2 * M->y[v];
        if (s != 0) tight = 0;
    }
    for (int i = 0; i < nbd; i++)
        if (q->BD[bl[i]] != m_rad(M, bl[i])) tight = 0;
    res->weight = wi / 2;
    res->obs = ob;
    res->primal_internal = wi;
    res->dual_sum = ds;
    res->dual_feasible = feas;
    res->tight = tight;
    res->events_implode += M->events[K_IMPLODE];
    res->events_collide += M->events[K_COLLIDE];
    res->events_boundary += M->events[K_BOUNDARY];
    free(pa); free(pb); free(bl);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: processing clusters from the detection events                 */
/* ------------------------------------------------------------------------- */

static int uf_find(int *p, int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/* level[a], cluster[a] (cluster ids 0.. in order of their lowest member). */
static int alg1_cluster(const Geo *q, int nlev, const long long *dk, const long long *bk,
                        int *level, int *cluster, int *nclusters) {
    int k = q->k;
    int *res = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    int *par = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    int *ok = (int *)malloc(sizeof(int) * (size_t)(k + 1));
    for (int a = 0; a < k; a++) { res[a] = 1; level[a] = 0; cluster[a] = -1; }
    int left = k, cid = 0;
    for (int lv = 0; lv < nlev && left > 0; lv++) {
        long long b = bk[lv], d = dk[lv];
        for (int a = 0; a < k; a++) par[a] = a;
        for (int a = 0; a < k; a++) {
            if (!res[a]) continue;
            for (int c = a + 1; c < k; c++)
                if (res[c] && q->D[a * k + c] <= b) {
                    int ra = uf_find(par, a), rc = uf_find(par, c);
                    if (ra != rc) par[ra < rc ? rc : ra] = ra < rc ? ra : rc;
                }
        }
        /* per component: diameter, size, boundary contact */
        for (int a = 0; a < k; a++) ok[a] = 0;
        for (int r = 0; r < k; r++) {
            if (!res[r] || uf_find(par, r) != r) continue;
            long long diam = 0;
            int size = 0, contact = 0;
            for (int a = 0; a < k; a++) {
                if (!res[a] || uf_find(par, a) != r) continue;
                size++;
                if (q->BD[a] < OR_INF && 2 * q->BD[a] <= b) contact = 1;
                for (int c = a + 1; c < k; c++)
                    if (res[c] && uf_find(par, c) == r && q->D[a * k + c] > diam) diam = q->D[a * k + c];
            }
            if (diam <= d && (contact || size % 2 == 0)) ok[r] = 1;
        }
        for (int r = 0; r < k; r++) {
            if (!res[r] || uf_find(par, r) != r || !ok[r]) continue;
            for (int a = 0; a < k; a++)
                if (res[a] && uf_find(par, a) == r) { level[a] = lv + 1; cluster[a] = cid; }
            cid++;
        }
        for (int a = 0; a < k; a++)
            if (res[a] && level[a] == lv + 1) { res[a] = 0; left--; }
    }
    *nclusters = cid;
    free(res); free(par); free(ok);
    return left == 0 ? ST_OK : ST_NO_SOLUTION;
}

/* ------------------------------------------------------------------------- */
/* Public entry points                                                        */
/* ------------------------------------------------------------------------- */

/* mode 0: global sparse blossom; mode 1: Alg. 1 + Alg. 2 hierarchical. */
int or_decode(const OGraph *g, int k, const int *det, int mode, int nlev,
              const long long *dk, const long long *bk, OResult *res, unsigned char *corr) {
    memset(res, 0, sizeof(*res));
    res->dual_feasible = 1;
    res->tight = 1;
    for (int i = 0; i < k; i++)
        if (det[i] < 0 || det[i] >= g->n || (i > 0 && det[i] <= det[i - 1])) return res->status = ST_BADARG;
    if (k == 0) {
        if (corr) memset(corr, 0, (size_t)g->m);
        return res->status = ST_OK;
    }
    Geo q;
    geo_build(g, k, det, &q);
    Matcher M;
    m_init(&M, &q);
    int st = ST_OK;
    if (mode == 0) {
        for (int a = 0; a < k; a++) m_add_root(&M, a);
        M.t = 0;
        st = m_run(&M);
        res->stop_time = M.t;
        res->e_ideal = M.nev;     /* one run: every event is on the critical path */
        res->t_ideal = M.t;
    } else {
        int *level = (int *)malloc(sizeof(int) * (size_t)k);
        int *cl = (int *)malloc(sizeof(int) * (size_t)k);
        int ncl = 0;
        st = alg1_cluster(&q, nlev, dk, bk, level, cl, &ncl);
        res->num_clusters = ncl;
        int maxlev = 0;
        for (int a = 0; a < k; a++) {
            if (level[a] > maxlev) maxlev = level[a];
            if (level[a] == 1) res->level1_events++;
        }
        res->num_levels = maxlev;
        int *cfg_level = (int *)calloc((size_t)ncl + 1, sizeof(int));
        /* Parallel event count (Methods, "Numerical evaluation"): t_lt and E_lt
         * are the critical-path stopping time and event count through the
         * levels below lv (both 0 below level 1).  A level-lv cluster C with
         * stopping time s(C) and event history E_C(t) (events at times <= t)
         * has t(C) = max(t_lt, s(C)) and
         *     E(C) = max(E_lt, E_C(t_lt)) + E_C(t(C)) - E_C(t_lt);
         * after the level, t_lt and E_lt become the maxima over its clusters
         * (unchanged if the level has none). */
        long long t_lt = 0, e_lt = 0;
        for (int lv = 1; st == ST_OK && lv <= maxlev; lv++) {
            long long t_next = t_lt, e_next = e_lt;
            for (int c = 0; st == ST_OK && c < ncl; c++) {
                int first = -1;
                for (int a = 0; a < k; a++)
                    if (cl[a] == c) { first = a; break; }
                if (first < 0 || level[first] != lv) continue;
                cfg_level[c] = lv;
                for (int v = 0; v < M.cap; v++) M.touched[v] = 0;
                for (int a = 0; a < k; a++)
                    if (cl[a] == c) { m_add_root(&M, a); M.config[a] = c; }
                M.t = 0;
                const long long ev0 = M.nev;
                st = m_run(&M);
                if (M.t > res->stop_time) res->stop_time = M.t;
                {
                    const long long s_c = M.t;                  /* time of the cluster's last event */
                    const long long n_c = M.nev - ev0;          /* E_C(t) for t >= s(C) */
                    long long n_below = 0;                      /* E_C(t_lt) */
                    for (long long i = ev0; i < M.nev; i++)
                        if (M.evt[i] <= t_lt) n_below++;
                    const long long t_c = s_c > t_lt ? s_c : t_lt;
                    const long long e_c = (e_lt > n_below ? e_lt : n_below) + n_c - n_below;
                    if (t_c > t_next) t_next = t_c;
                    if (e_c > e_next) e_next = e_c;
                }
                /* touched retained configurations join cluster c's configuration */
                int *hit = (int *)calloc((size_t)ncl + 1, sizeof(int));
                for (int v = 0; v < M.nnodes; v++)
                    if (M.touched[v] && M.config[v] >= 0 && M.config[v] != c) hit[M.config[v]] = 1;
                for (int o = 0; o < ncl; o++) {
                    if (!hit[o]) continue;
                    if (cfg_level[o] >= lv) res->touch_violations++;
                    for (int v = 0; v < M.cap; v++)
                        if (M.config[v] == o) M.config[v] = c;
                }
                for (int v = 0; v < M.cap; v++)
                    if (M.alive[v] && M.touched[v] && M.config[v] < 0) M.config[v] = c;
                free(hit);
            }
            t_lt = t_next;
            e_lt = e_next;
        }
        res->e_ideal = e_lt;
        res->t_ideal = t_lt;
        free(cfg_level); free(level); free(cl);
    }
    if (st == ST_OK) m_finish(&M, res, g, corr);
    res->events_implode = M.events[K_IMPLODE];
    res->events_collide = M.events[K_COLLIDE];
    res->events_boundary = M.events[K_BOUNDARY];
    m_free(&M);
    geo_free(&q);
    return res->status = st;
}

/* Decode a block of shots given as padded uint32 bitmaps (LSB-first). */
int or_decode_bitmaps(const OGraph *g, long long nshots, int words, const uint32_t *syn, int mode,
                      int nlev, const long long *dk, const long long *bk,
                      long long *weight, uint64_t *obs, int *status) {
    int *det = (int *)malloc(sizeof(int) * (size_t)(g->n + 1));
    for (long long s = 0; s < nshots; s++) {
        const uint32_t *row = syn + s * (long long)words;
        int k = 0;
        for (int x = 0; x < g->n; x++)
            if ((row[x >> 5] >> (x & 31)) & 1u) det[k++] = x;
        OResult r;
        or_decode(g, k, det, mode, nlev, dk, bk, &r, NULL);
        weight[s] = r.weight;
        obs[s] = r.obs;
        status[s] = r.status;
    }
    free(det);
    return ST_OK;
}

/* Exact geometry of one shot, for the tests. */
void or_geometry(const OGraph *g, int k, const int *det, long long *D, uint64_t *PO, long long *BD,
                 int *BE, uint64_t *BO) {
    Geo q;
    geo_build(g, k, det, &q);
    memcpy(D, q.D, sizeof(long long) * (size_t)(k * k));
    memcpy(PO, q.PO, sizeof(uint64_t) * (size_t)(k * k));
    memcpy(BD, q.BD, sizeof(long long) * (size_t)k);
    memcpy(BE, q.BE, sizeof(int) * (size_t)k);
    memcpy(BO, q.BO, sizeof(uint64_t) * (size_t)k);
    geo_free(&q);
}

/* Algorithm 1 alone, for the tests. */
int or_cluster(const OGraph *g, int k, const int *det, int nlev, const long long *dk,
               const long long *bk, int *level, int *cluster) {
    Geo q;
    geo_build(g, k, det, &q);
    int nc = 0;
    int st = alg1_cluster(&q, nlev, dk, bk, level, cluster, &nc);
    geo_free(&q);
    return st;
}

int or_result_size(void) { return (int)sizeof(OResult); }
