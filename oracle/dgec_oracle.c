/*
 * dgec oracle -- plain, slow, single-threaded CPU restatement of the method of
 * "Scalable Edge Clustering of Dynamic Graphs via Weighted Line Graphs"
 * (arXiv 2311.10337).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (each reading of the paper is listed where it is used):
 *   - temporal edge e = (src[e], dst[e], t[e]); its id is its input position;
 *     ids are the nodes of the line graph.
 *   - all arithmetic is integer; nothing here is floating point.
 *
 * Parity pins: every function below is pinned by tests in tests/ against
 * brute force on the explicit line graph (Def. 1), against Thm. 1-3, and
 * against the worked example printed in the paper (the chain table of
 * Sec. 4.1.3). The condensed-tree / excess-of-mass step of Alg. 1
 * is defined by the paper only by citation to HDBSCAN; its pins are the
 * hand-worked golden cases under tests/golden/ and filtration invariants.
 * The discrete dendrogram (Alg. 5) is pinned against brute-force components
 * of the explicit line graph at every threshold; condensing it is pinned by
 * reduction to the continuous condense (one threshold per distinct weight,
 * and weights rounded up to coarse thresholds) and by a closed form for one
 * level.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_VERTEX 2
#define ORC_ERR_SELF_LOOP 3
#define ORC_ERR_OOM 5

/* ------------------------------------------------------------------ */
/* Incidence lists (the adjacency lists of G that Alg. 3 starts from).  */
/* Each vertex keeps its in-list and out-list sorted by (t, id)        */
/* (Alg. 2's time order; ties by id, a reading).                       */
/* ------------------------------------------------------------------ */

static const int64_t *g_t; /* comparator context */

static int cmp_by_time_then_id(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_t[x] != g_t[y]) return g_t[x] < g_t[y] ? -1 : 1;
    return (x > y) - (x < y);
}

int orc_validate(int64_t n_edges, int32_t n_vertices, const int32_t *src,
                 const int32_t *dst)
{
    if (n_edges < 0 || n_vertices < 0) return ORC_ERR_ARG;
    for (int64_t e = 0; e < n_edges; e++) {
        if (src[e] < 0 || src[e] >= n_vertices || dst[e] < 0 || dst[e] >= n_vertices)
            return ORC_ERR_VERTEX;
        if (src[e] == dst[e]) return ORC_ERR_SELF_LOOP; /* Sec. 1.2.1: no self loops */
    }
    return ORC_OK;
}

/* out_off/in_off: n_vertices+1 entries; out_id/in_id: n_edges entries. */
int orc_csr(int64_t n_edges, int32_t n_vertices, const int32_t *src,
            const int32_t *dst, const int64_t *t, int64_t *out_off,
            int32_t *out_id, int64_t *in_off, int32_t *in_id)
{
    int rc = orc_validate(n_edges, n_vertices, src, dst);
    if (rc) return rc;
    memset(out_off, 0, sizeof(int64_t) * ((size_t)n_vertices + 1));
    memset(in_off, 0, sizeof(int64_t) * ((size_t)n_vertices + 1));
    for (int64_t e = 0; e < n_edges; e++) {
        out_off[src[e] + 1]++;
        in_off[dst[e] + 1]++;
    }
    for (int32_t v = 0; v < n_vertices; v++) {
        out_off[v + 1] += out_off[v];
        in_off[v + 1] += in_off[v];
    }
    int64_t *fo = malloc(sizeof(int64_t) * ((size_t)n_vertices + 1));
    int64_t *fi = malloc(sizeof(int64_t) * ((size_t)n_vertices + 1));
    if (!fo || !fi) { free(fo); free(fi); return ORC_ERR_OOM; }
    memcpy(fo, out_off, sizeof(int64_t) * ((size_t)n_vertices + 1));
    memcpy(fi, in_off, sizeof(int64_t) * ((size_t)n_vertices + 1));
    for (int64_t e = 0; e < n_edges; e++) {
        out_id[fo[src[e]]++] = (int32_t)e;
        in_id[fi[dst[e]]++] = (int32_t)e;
    }
    free(fo);
    free(fi);
    g_t = t;
    for (int32_t v = 0; v < n_vertices; v++) {
        qsort(out_id + out_off[v], (size_t)(out_off[v + 1] - out_off[v]),
              sizeof(int32_t), cmp_by_time_then_id);
        qsort(in_id + in_off[v], (size_t)(in_off[v + 1] - in_off[v]),
              sizeof(int32_t), cmp_by_time_then_id);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 2 (node-local MST of the line graph) and Alg. 3 (skeleton).     */
/* ------------------------------------------------------------------ */

typedef struct { int64_t t; int32_t dir; int32_t id; } inc_rec; /* dir: 0 in, 1 out */

static int cmp_inc(const void *a, const void *b)
{
    const inc_rec *x = a, *y = b;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    /* Reading: at equal times an in-edge precedes an out-edge. P2 is
     * non-strict (Def. 1) and the perturbation in the proof of Thm. 2
     * (t'_q = t_q + gamma q > t'_p = t_p + gamma^2 p) puts in before out. */
    if (x->dir != y->dir) return x->dir - y->dir;
    return (x->id > y->id) - (x->id < y->id);
}

/*
 * Raw output of Alg. 2 run at every vertex i (Alg. 3's loop), in emission
 * order: (in-edge p, out-edge q, w = t_q - t_p, centre vertex i).
 * Capacity: 2 * n_edges records. Returns the count, or -1 on bad input.
 */
int64_t orc_skeleton_raw(int64_t n_edges, int32_t n_vertices,
                         const int32_t *src, const int32_t *dst,
                         const int64_t *t, int32_t *p_out, int32_t *q_out,
                         int64_t *w_out, int32_t *centre_out)
{
    if (orc_validate(n_edges, n_vertices, src, dst)) return -1;
    int64_t *deg = calloc((size_t)n_vertices + 1, sizeof(int64_t));
    if (!deg) return -1;
    for (int64_t e = 0; e < n_edges; e++) { deg[src[e] + 1]++; deg[dst[e] + 1]++; }
    for (int32_t v = 0; v < n_vertices; v++) deg[v + 1] += deg[v];
    inc_rec *all = malloc(sizeof(inc_rec) * (size_t)(2 * n_edges + 1));
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)n_vertices + 1));
    int32_t *W = malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    if (!all || !fill || !W) { free(deg); free(all); free(fill); free(W); return -1; }
    memcpy(fill, deg, sizeof(int64_t) * ((size_t)n_vertices + 1));
    for (int64_t e = 0; e < n_edges; e++) {
        inc_rec r;
        r.t = t[e]; r.id = (int32_t)e;
        r.dir = 1; all[fill[src[e]]++] = r; /* e leaves src[e] */
        r.dir = 0; all[fill[dst[e]]++] = r; /* e enters dst[e] */
    }
    int64_t n_out = 0;
    for (int32_t i = 0; i < n_vertices; i++) {
        inc_rec *Ei = all + deg[i];
        int64_t di = deg[i + 1] - deg[i];
        qsort(Ei, (size_t)di, sizeof(inc_rec), cmp_inc); /* Alg. 2: E_i in time order */
        int64_t wlen = 0;                                /* W = [] */
        for (int64_t x = 0; x < di; x++) {
            if (Ei[x].dir == 0) {
                W[wlen++] = Ei[x].id;                    /* W.append(e_j) */
            } else {
                for (int64_t y = 0; y < wlen; y++) {     /* output (e_k, e_j) */
                    p_out[n_out] = W[y];
                    q_out[n_out] = Ei[x].id;
                    w_out[n_out] = Ei[x].t - t[W[y]];    /* P3: w = t_s - t_r */
                    centre_out[n_out] = i;
                    n_out++;
                }
                /* W = [W[-1]]; reading: an empty W stays empty. */
                if (wlen > 0) { W[0] = W[wlen - 1]; wlen = 1; }
            }
        }
    }
    free(deg); free(all); free(fill); free(W);
    return n_out;
}

typedef struct { int64_t w; int32_t u; int32_t v; } wedge;

static int cmp_wedge(const void *a, const void *b)
{
    const wedge *x = a, *y = b;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    return (x->v > y->v) - (x->v < y->v);
}

/*
 * Skeleton L*_G = union over vertices of M_G(i) (Alg. 3), as an undirected
 * edge set: each line-graph edge is written (u = min id, v = max id, w);
 * the union is a set, so repeated (u, v, w) are kept once; sorted by
 * (w, u, v). Capacity 2 * n_edges. Returns the count or -1.
 */
int64_t orc_skeleton(int64_t n_edges, int32_t n_vertices, const int32_t *src,
                     const int32_t *dst, const int64_t *t, int32_t *u_out,
                     int32_t *v_out, int64_t *w_out)
{
    size_t cap = (size_t)(2 * n_edges + 1);
    int32_t *p = malloc(sizeof(int32_t) * cap), *q = malloc(sizeof(int32_t) * cap);
    int32_t *c = malloc(sizeof(int32_t) * cap);
    int64_t *w = malloc(sizeof(int64_t) * cap);
    wedge *all = malloc(sizeof(wedge) * cap);
    if (!p || !q || !c || !w || !all) { free(p); free(q); free(c); free(w); free(all); return -1; }
    int64_t n = orc_skeleton_raw(n_edges, n_vertices, src, dst, t, p, q, w, c);
    if (n < 0) { free(p); free(q); free(c); free(w); free(all); return -1; }
    for (int64_t x = 0; x < n; x++) {
        all[x].w = w[x];
        all[x].u = p[x] < q[x] ? p[x] : q[x];
        all[x].v = p[x] < q[x] ? q[x] : p[x];
    }
    qsort(all, (size_t)n, sizeof(wedge), cmp_wedge);
    int64_t m = 0;
    for (int64_t x = 0; x < n; x++) {
        if (m > 0 && cmp_wedge(&all[m - 1], &all[x]) == 0) continue;
        all[m++] = all[x];
    }
    for (int64_t x = 0; x < m; x++) { u_out[x] = all[x].u; v_out[x] = all[x].v; w_out[x] = all[x].w; }
    free(p); free(q); free(c); free(w); free(all);
    return m;
}

/* ------------------------------------------------------------------ */
/* k nearest line-graph neighbours in time and core distance.          */
/* Reading: in the undirected line graph of Def. 1, the neighbours of  */
/* e = (i, j, t_e) are the in-edges r of i with t_r <= t_e (arc r->e)  */
/* and the out-edges s of j with t_s >= t_e (arc e->s); weight |dt|.   */
/* Neighbours are ranked by (w, id), repeated ids kept once; core(e)  */
/* is the weight of the k-th, or INT64_MAX if fewer than k exist.     */
/* ------------------------------------------------------------------ */

typedef struct { int64_t w; int32_t id; } cand;

static int cmp_cand(const void *a, const void *b)
{
    const cand *x = a, *y = b;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Queries: n_query edge ids; knn_out[n_query * k], core_out[n_query].
 * dmax: the time cutoff of Sec. 4.3 -- only arcs with w <= dmax are in
 * the line graph, so only such neighbours count (INT64_MAX: no cutoff).
 * dnc: the nearly-causal tolerance of Sec. 4.3 -- an arc r -> s also
 * exists when s is at most dnc earlier than r (t_s >= t_r - dnc), weighed
 * |t_s - t_r| (0: the causal line graph of Def. 1). */
int orc_knn(int64_t n_edges, int32_t n_vertices, const int32_t *src,
            const int32_t *dst, const int64_t *t, int32_t k,
            int64_t n_query, const int32_t *query, int64_t dmax, int64_t dnc,
            int32_t *knn_out, int64_t *core_out)
{
    if (k < 1) return ORC_ERR_ARG;
    int64_t *out_off = malloc(sizeof(int64_t) * ((size_t)n_vertices + 1));
    int64_t *in_off = malloc(sizeof(int64_t) * ((size_t)n_vertices + 1));
    int32_t *out_id = malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    int32_t *in_id = malloc(sizeof(int32_t) * (size_t)(n_edges + 1));
    if (!out_off || !in_off || !out_id || !in_id) return ORC_ERR_OOM;
    int rc = orc_csr(n_edges, n_vertices, src, dst, t, out_off, out_id, in_off, in_id);
    if (rc) { free(out_off); free(in_off); free(out_id); free(in_id); return rc; }
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n_vertices; v++) {
        int64_t a = in_off[v + 1] - in_off[v], b = out_off[v + 1] - out_off[v];
        if (a > maxdeg) maxdeg = a;
        if (b > maxdeg) maxdeg = b;
    }
    cand *c = malloc(sizeof(cand) * (size_t)(2 * maxdeg + 2));
    if (!c) return ORC_ERR_OOM;
    for (int64_t qx = 0; qx < n_query; qx++) {
        int32_t e = query[qx];
        int32_t i = src[e], j = dst[e];
        int64_t nc = 0;
        for (int64_t x = in_off[i]; x < in_off[i + 1]; x++) {   /* predecessors */
            int32_t r = in_id[x];
            int64_t d = t[e] - t[r];                             /* arc r -> e: t_e >= t_r - dnc */
            int64_t w = d < 0 ? -d : d;
            if (d >= -dnc && w <= dmax) { c[nc].w = w; c[nc].id = r; nc++; }
        }
        for (int64_t x = out_off[j]; x < out_off[j + 1]; x++) { /* successors */
            int32_t s = out_id[x];
            int64_t d = t[s] - t[e];                             /* arc e -> s: t_s >= t_e - dnc */
            int64_t w = d < 0 ? -d : d;
            if (d >= -dnc && w <= dmax) { c[nc].w = w; c[nc].id = s; nc++; }
        }
        qsort(c, (size_t)nc, sizeof(cand), cmp_cand);
        int32_t got = 0;
        int64_t last_w = INT64_MAX;
        for (int64_t x = 0; x < nc && got < k; x++) {
            if (x > 0 && c[x].id == c[x - 1].id) continue; /* same node via both arcs */
            knn_out[qx * k + got] = c[x].id;
            last_w = c[x].w;
            got++;
        }
        for (int32_t y = got; y < k; y++) knn_out[qx * k + y] = -1;
        core_out[qx] = (got == k) ? last_w : INT64_MAX;
    }
    free(c); free(out_off); free(in_off); free(out_id); free(in_id);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 1, spanning forest: minimum spanning forest by Kruskal on the  */
/* undirected skeleton, edges taken in (w, u, v) order (a strict       */
/* total order, so the forest is unique).                             */
/* ------------------------------------------------------------------ */

static int32_t uf_find(int32_t *par, int32_t x)
{
    int32_t r = x;
    while (par[r] != r) r = par[r];
    while (par[x] != r) { int32_t nx = par[x]; par[x] = r; x = nx; }
    return r;
}

/* Skeleton edges in any order; output the forest sorted by (w, u, v). */
int64_t orc_mst(int64_t n_nodes, int64_t n_sk, const int32_t *u,
                const int32_t *v, const int64_t *w, int32_t *mu, int32_t *mv,
                int64_t *mw)
{
    wedge *all = malloc(sizeof(wedge) * (size_t)(n_sk + 1));
    int32_t *par = malloc(sizeof(int32_t) * (size_t)(n_nodes + 1));
    if (!all || !par) { free(all); free(par); return -1; }
    for (int64_t x = 0; x < n_sk; x++) {
        all[x].w = w[x];
        all[x].u = u[x] < v[x] ? u[x] : v[x];
        all[x].v = u[x] < v[x] ? v[x] : u[x];
    }
    qsort(all, (size_t)n_sk, sizeof(wedge), cmp_wedge); /* Alg. 1's weight order */
    for (int64_t x = 0; x < n_nodes; x++) par[x] = (int32_t)x;
    int64_t m = 0;
    for (int64_t x = 0; x < n_sk; x++) {
        int32_t a = uf_find(par, all[x].u), b = uf_find(par, all[x].v);
        if (a == b) continue;
        par[a] = b;
        mu[m] = all[x].u; mv[m] = all[x].v; mw[m] = all[x].w; m++;
    }
    free(all); free(par);
    return m;
}

/* ------------------------------------------------------------------ */
/* Alg. 1, dendrogram: union-find replay of the sorted forest.         */
/* Row s merges the clusters holding mu[s] and mv[s]; a cluster is     */
/* named by a leaf id (< n_nodes) or n_nodes + (row that formed it).   */
/* a = smaller name, b = larger name, size = leaves below the row.     */
/* ------------------------------------------------------------------ */

int orc_linkage(int64_t n_nodes, int64_t n_mst, const int32_t *mu,
                const int32_t *mv, int32_t *a_out, int32_t *b_out,
                int64_t *size_out)
{
    int32_t *par = malloc(sizeof(int32_t) * (size_t)(n_nodes + 1));
    int32_t *name = malloc(sizeof(int32_t) * (size_t)(n_nodes + 1));
    int64_t *sz = malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
    if (!par || !name || !sz) { free(par); free(name); free(sz); return ORC_ERR_OOM; }
    for (int64_t x = 0; x < n_nodes; x++) { par[x] = (int32_t)x; name[x] = (int32_t)x; sz[x] = 1; }
    for (int64_t s = 0; s < n_mst; s++) {
        int32_t ra = uf_find(par, mu[s]), rb = uf_find(par, mv[s]);
        int32_t na = name[ra], nb = name[rb];
        a_out[s] = na < nb ? na : nb;
        b_out[s] = na < nb ? nb : na;
        size_out[s] = sz[ra] + sz[rb];
        par[ra] = rb;
        sz[rb] += sz[ra];
        name[rb] = (int32_t)(n_nodes + s);
    }
    free(par); free(name); free(sz);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 1, condensing and extraction: condensed tree with minimum      */
/* cluster size M and excess-of-mass cluster selection (the paper's    */
/* volume in dendrogram space).                                       */
/* The paper defines these steps by citation to HDBSCAN; readings:     */
/*  - merges of equal weight are one multi-way merge (level collapse), */
/*    so the result depends only on the weighted connectivity;         */
/*  - lambda(w) = floor((2^64 - 1) / (w + 1)) as an unsigned integer, */
/*    and lambda = 0 at a virtual root of weight infinity whose        */
/*    children are the components;                                     */
/*  - stabilities are exact 128-bit integers; EOM ties go to the parent;*/
/*    the root cluster is never selected;                              */
/*  - labels: -1 for noise, clusters numbered by their smallest id.    */
/* ------------------------------------------------------------------ */

typedef unsigned __int128 u128;

static uint64_t lam(int64_t w) { return UINT64_MAX / ((uint64_t)w + 1u); }

/*
 * Inputs: linkage rows (a, b, w, size), n_mst rows over n_nodes leaves.
 * Outputs (caller allocates):
 *   fall_cluster[n_nodes], fall_lambda[n_nodes]: cluster each point leaves
 *     and the lambda at which it leaves;
 *   cl_id, cl_parent, cl_birth, cl_death, cl_size, cl_stab_hi, cl_stab_lo,
 *   cl_selected[n_nodes + 1 max]: clusters sorted by id (the node id of the
 *     merge that starts them; the root cluster's id is n_nodes + n_mst);
 *     cl_death = 0 for clusters that never split; cl_parent = -1 for root;
 *     cl_selected: 1 selected by EOM (before removing descendants of
 *     selected ones), 2 in the final selection, 0 otherwise;
 *   labels[n_nodes]; returns the number of clusters written to *n_cl and
 *   the number of final clusters to *n_labels.
 */
int orc_condense(int64_t n_nodes, int64_t n_mst, const int32_t *a,
                 const int32_t *b, const int64_t *w, const int64_t *size,
                 int32_t M, int32_t *fall_cluster, uint64_t *fall_lambda,
                 int32_t *cl_id, int32_t *cl_parent, uint64_t *cl_birth,
                 uint64_t *cl_death, int64_t *cl_size, uint64_t *cl_stab_hi,
                 uint64_t *cl_stab_lo, int32_t *cl_selected, int32_t *labels,
                 int64_t *n_cl, int32_t *n_labels)
{
    if (M < 2) return ORC_ERR_ARG;
    int64_t n_all = n_nodes + n_mst + 1;          /* leaves, merges, virtual root */
    int32_t root = (int32_t)(n_nodes + n_mst);
    int32_t *parent = malloc(sizeof(int32_t) * (size_t)n_all);
    int32_t *cpar = malloc(sizeof(int32_t) * (size_t)n_all);   /* collapsed parent */
    int64_t *nsize = malloc(sizeof(int64_t) * (size_t)n_all);
    int64_t *coff = calloc((size_t)n_all + 1, sizeof(int64_t));
    int32_t *kids = malloc(sizeof(int32_t) * (size_t)n_all);
    int32_t *node_cl = malloc(sizeof(int32_t) * (size_t)n_all);   /* cluster a node stands for */
    int32_t *stack = malloc(sizeof(int32_t) * (size_t)n_all);
    int32_t *cl_of = malloc(sizeof(int32_t) * (size_t)n_all);     /* cluster id -> row */
    u128 *stab = calloc((size_t)n_all, sizeof(u128));
    u128 *S = calloc((size_t)n_all, sizeof(u128));
    int32_t *minmem = malloc(sizeof(int32_t) * (size_t)n_all);
    if (!parent || !cpar || !nsize || !coff || !kids || !node_cl || !stack ||
        !cl_of || !stab || !S || !minmem)
        return ORC_ERR_OOM;

    for (int64_t x = 0; x < n_all; x++) parent[x] = -1;
    for (int64_t x = 0; x < n_nodes; x++) nsize[x] = 1;
    for (int64_t s = 0; s < n_mst; s++) {
        parent[a[s]] = (int32_t)(n_nodes + s);
        parent[b[s]] = (int32_t)(n_nodes + s);
        nsize[n_nodes + s] = size[s];
    }
    nsize[root] = n_nodes;
    /* A merge node is kept ("representative") when its parent has another
     * weight or it has no parent; equal-weight chains fold into their top. */
#define NODE_W(x) (w[(x) - n_nodes])
    /* top[x]: highest merge reachable from merge x through parents of the
     * same weight; parents have larger ids, so a descending sweep sees a
     * parent before its children. */
    int32_t *top = malloc(sizeof(int32_t) * (size_t)n_all);
    if (!top) return ORC_ERR_OOM;
    for (int64_t x = n_nodes + n_mst - 1; x >= n_nodes; x--) {
        int32_t p = parent[x];
        top[x] = (p >= 0 && NODE_W(p) == NODE_W(x)) ? top[p] : (int32_t)x;
    }
    for (int64_t x = 0; x < n_all - 1; x++)
        cpar[x] = parent[x] < 0 ? root : top[parent[x]];
    cpar[root] = -1;
    free(top);
    /* children lists of kept nodes (leaves and representatives) */
    for (int64_t x = 0; x < n_all - 1; x++) {
        int keep = (x < n_nodes) || parent[x] < 0 || NODE_W(parent[x]) != NODE_W(x);
        if (keep) coff[cpar[x] + 1]++;
    }
    for (int64_t x = 0; x < n_all; x++) coff[x + 1] += coff[x];
    {
        int64_t *f = malloc(sizeof(int64_t) * (size_t)n_all);
        memcpy(f, coff, sizeof(int64_t) * (size_t)n_all);
        for (int64_t x = 0; x < n_all - 1; x++) {
            int keep = (x < n_nodes) || parent[x] < 0 || NODE_W(parent[x]) != NODE_W(x);
            if (keep) kids[f[cpar[x]]++] = (int32_t)x;
        }
        free(f);
    }
    /* lambda of a kept node: lambda(w), 0 for the virtual root */
#define NODE_L(x) ((x) == root ? 0u : lam(NODE_W(x)))

    int64_t ncl = 0;
    for (int64_t x = 0; x < n_all; x++) { node_cl[x] = -1; cl_of[x] = -1; }
    /* clusters are created in a top-down walk; per-cluster scratch: */
    int32_t *cparent = malloc(sizeof(int32_t) * (size_t)n_all);
    uint64_t *cbirth = malloc(sizeof(uint64_t) * (size_t)n_all);
    uint64_t *cdeath = calloc((size_t)n_all, sizeof(uint64_t));
    int64_t *csize = malloc(sizeof(int64_t) * (size_t)n_all);
    int32_t *sel = calloc((size_t)n_all, sizeof(int32_t));
    if (!cparent || !cbirth || !cdeath || !csize || !sel) return ORC_ERR_OOM;
    /* root cluster */
    cparent[root] = -1; cbirth[root] = 0; csize[root] = n_nodes;
    node_cl[root] = root;
    int64_t sp = 0;
    stack[sp++] = root;
    int32_t *leafstack = malloc(sizeof(int32_t) * (size_t)n_all);
    while (sp > 0) {
        int32_t X = stack[--sp];
        int32_t K = node_cl[X];
        uint64_t LX = NODE_L(X);
        int64_t nbig = 0;
        for (int64_t y = coff[X]; y < coff[X + 1]; y++)
            if (nsize[kids[y]] >= M) nbig++;
        if (nbig >= 2) cdeath[K] = LX;                  /* K splits here */
        for (int64_t y = coff[X]; y < coff[X + 1]; y++) {
            int32_t c = kids[y];
            if (nsize[c] >= M) {
                if (nbig >= 2) {                        /* new cluster born at LX */
                    node_cl[c] = c;
                    cparent[c] = K; cbirth[c] = LX; csize[c] = nsize[c];
                } else {
                    node_cl[c] = K;                     /* the only big child continues K */
                }
                stack[sp++] = c;
            } else {
                /* every point under a small child leaves K at LX */
                int64_t lp = 0;
                leafstack[lp++] = c;
                while (lp > 0) {
                    int32_t z = leafstack[--lp];
                    if (z < n_nodes) {
                        fall_cluster[z] = K;
                        fall_lambda[z] = LX;
                    } else {
                        for (int64_t q = coff[z]; q < coff[z + 1]; q++) leafstack[lp++] = kids[q];
                    }
                }
            }
        }
    }
    free(leafstack);
    /* stabilities (exact): sum over points of (lambda_leave - lambda_birth) */
    for (int64_t p = 0; p < n_nodes; p++) {
        int32_t K = fall_cluster[p];
        stab[K] += (u128)(fall_lambda[p] - cbirth[K]);
    }
    /* child clusters: their points leave the parent at the parent's death */
    int32_t *clist = malloc(sizeof(int32_t) * (size_t)n_all);
    for (int64_t x = 0; x < n_all; x++)
        if (node_cl[x] == (int32_t)x) clist[ncl++] = (int32_t)x;   /* ascending id */
    for (int64_t c = 0; c < ncl; c++) {
        int32_t K = clist[c];
        if (cparent[K] >= 0) {
            int32_t P = cparent[K];
            stab[P] += (u128)csize[K] * (u128)(cdeath[P] - cbirth[P]);
        }
    }
    /* excess of mass, bottom-up: a child cluster's id is always smaller
     * than its parent's (it is born at a descendant merge), so ascending
     * id order visits children first. */
    u128 *childsum = calloc((size_t)n_all, sizeof(u128));
    for (int64_t c = 0; c < ncl; c++) {
        int32_t K = clist[c];
        if (K == root) continue;
        if (stab[K] >= childsum[K]) { sel[K] = 1; S[K] = stab[K]; }
        else { sel[K] = 0; S[K] = childsum[K]; }
        childsum[cparent[K]] += S[K];
    }
    free(childsum);
    /* final selection: selected with no selected ancestor below the root.
     * fin[K] = the final cluster on the path from K up (or -1); a parent
     * has a larger id, so a descending sweep fills parents first. */
    int32_t *fin = malloc(sizeof(int32_t) * (size_t)n_all);
    if (!fin) return ORC_ERR_OOM;
    for (int64_t c = ncl - 1; c >= 0; c--) {
        int32_t K = clist[c];
        if (K == root) { fin[K] = -1; continue; }
        int32_t up = fin[cparent[K]];
        if (up >= 0) fin[K] = up;
        else if (sel[K]) { sel[K] = 2; fin[K] = K; }
        else fin[K] = -1;
    }
    /* labels: the final cluster on the path from the point's cluster up */
    for (int64_t x = 0; x < n_all; x++) minmem[x] = INT32_MAX;
    for (int64_t p = 0; p < n_nodes; p++) {
        int32_t lab = fin[fall_cluster[p]];
        labels[p] = lab;
        if (lab >= 0 && (int32_t)p < minmem[lab]) minmem[lab] = (int32_t)p;
    }
    free(fin);
    /* number final clusters by smallest member id */
    int32_t nlab = 0;
    int32_t *rankof = malloc(sizeof(int32_t) * (size_t)n_all);
    for (int64_t x = 0; x < n_all; x++) rankof[x] = -1;
    for (int64_t p = 0; p < n_nodes; p++) {      /* ascending p meets each min first */
        int32_t L = labels[p];
        if (L >= 0 && minmem[L] == (int32_t)p) rankof[L] = nlab++;
    }
    for (int64_t p = 0; p < n_nodes; p++)
        if (labels[p] >= 0) labels[p] = rankof[labels[p]];
    for (int64_t c = 0; c < ncl; c++) {
        int32_t K = clist[c];
        cl_id[c] = K;
        cl_parent[c] = cparent[K];
        cl_birth[c] = cbirth[K];
        cl_death[c] = cdeath[K];
        cl_size[c] = csize[K];
        cl_stab_hi[c] = (uint64_t)(stab[K] >> 64);
        cl_stab_lo[c] = (uint64_t)stab[K];
        cl_selected[c] = (K == root) ? 0 : sel[K];
    }
    *n_cl = ncl;
    *n_labels = nlab;
    free(parent); free(cpar); free(nsize); free(coff); free(kids); free(node_cl);
    free(stack); free(cl_of); free(stab); free(S); free(minmem); free(cparent);
    free(cbirth); free(cdeath); free(csize); free(sel); free(clist); free(rankof);
    return ORC_OK;
#undef NODE_W
#undef NODE_L
}

/* ------------------------------------------------------------------ */
/* Alg. 5: discrete dendrogram. For each threshold omega_i (increasing),  */
/* comps(H, omega_i) of the graph H restricted to edges of weight         */
/* <= omega_i (reading: "<=" as in the appendix). Level i of the output   */
/* names every node's component by its smallest member id; the tree D     */
/* follows from the labels (component c at level i-1 has parent           */
/* labels[i][c] at level i).                                              */
/* ------------------------------------------------------------------ */

static int32_t uf_find_min(int32_t *par, int32_t x)
{
    int32_t r = x;
    while (par[r] != r) r = par[r];
    while (par[x] != r) { int32_t nx = par[x]; par[x] = r; x = nx; }
    return r;
}

int orc_levels(int64_t n_nodes, int64_t n_edges, const int32_t *u, const int32_t *v,
               const int64_t *w, int32_t q, const int64_t *omega, int32_t *labels)
{
    int32_t *par = malloc(sizeof(int32_t) * (size_t)(n_nodes + 1));
    if (!par) return ORC_ERR_OOM;
    for (int32_t i = 0; i < q; i++) {
        /* comps(H, omega_i), computed afresh for every threshold */
        for (int64_t x = 0; x < n_nodes; x++) par[x] = (int32_t)x;
        for (int64_t e = 0; e < n_edges; e++) {
            if (w[e] > omega[i]) continue;
            int32_t a = uf_find_min(par, u[e]), b = uf_find_min(par, v[e]);
            if (a == b) continue;
            if (a < b) par[b] = a; else par[a] = b;   /* smaller id stays the root */
        }
        for (int64_t x = 0; x < n_nodes; x++) labels[(int64_t)i * n_nodes + x] = uf_find_min(par, (int32_t)x);
    }
    free(par);
    return ORC_OK;
}

/* The tree D of Alg. 5 in per-node form. Every component at threshold i is
 * named by its smallest member, so a node x names a component from level 0
 * up to the first level at which a smaller node joins its component; there
 * the containment edge (x's component at level i-1) -> (its component at
 * level i) is recorded as merge_level[x] = i, merge_parent[x] = the name of
 * the level-i component. Nodes that name a component at every level get
 * -1, -1. Levels are 0-based; "level -1" is the singletons. */
int orc_levels_tree(int64_t n_nodes, int32_t q, const int32_t *labels,
                    int32_t *merge_level, int32_t *merge_parent)
{
    for (int64_t x = 0; x < n_nodes; x++) {
        merge_level[x] = -1;
        merge_parent[x] = -1;
        for (int32_t i = 0; i < q; i++) {
            int32_t c = labels[(int64_t)i * n_nodes + x];
            if (c != (int32_t)x) { merge_level[x] = i; merge_parent[x] = c; break; }
        }
    }
    return ORC_OK;
}

/* Step 4-5 of Alg. 1 on the discrete dendrogram D (Sec. 3, condensing on
 * the discrete dendrogram): the HDBSCAN condensed tree, stabilities and
 * excess-of-mass selection, walked top-down over D's nodes. Nodes of D:
 * the singletons x (id x), the components (i, c) of level i (id
 * (i + 1) * n + c, c = smallest member) and a virtual root above the last
 * level (id (q + 1) * n, lambda 0). Going down from a level-i node, its
 * children are the level-(i-1) components inside it; the event happens at
 * lambda(omega_i) = floor((2^64 - 1) / (omega_i + 1)). Conventions as in
 * orc_condense: a cluster splits when two or more children have >= M
 * members, the only big child otherwise carries the cluster on, small
 * children's points fall out; stabilities in exact 128-bit arithmetic;
 * the root is never selected; labels numbered by smallest member. The
 * cluster table lists clusters in ascending node id. */
int orc_condense_levels(int64_t n, int32_t q, const int64_t *omega,
                        const int32_t *lab, int32_t M, int32_t *labels,
                        int32_t *n_labels, int64_t *n_cl, uint64_t *cl_birth,
                        uint64_t *cl_death, int64_t *cl_size, uint64_t *cl_stab_hi,
                        uint64_t *cl_stab_lo, int32_t *cl_selected)
{
    if (M < 2 || q < 1) return ORC_ERR_ARG;
    int64_t N = (int64_t)(q + 1) * n + 1;
    int64_t root = N - 1;
    char *exists = calloc((size_t)N, 1);
    int64_t *parent = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *nsize = calloc((size_t)N, sizeof(int64_t));
    int64_t *coff = calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *kids = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *node_cl = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *leafstack = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *cparent = malloc(sizeof(int64_t) * (size_t)N);
    uint64_t *cbirth = calloc((size_t)N, sizeof(uint64_t));
    uint64_t *cdeath = calloc((size_t)N, sizeof(uint64_t));
    int64_t *csize = calloc((size_t)N, sizeof(int64_t));
    int32_t *sel = calloc((size_t)N, sizeof(int32_t));
    u128 *stab = calloc((size_t)N, sizeof(u128));
    u128 *S = calloc((size_t)N, sizeof(u128));
    u128 *childsum = calloc((size_t)N, sizeof(u128));
    int64_t *fall_cluster = malloc(sizeof(int64_t) * (size_t)(n + 1));
    uint64_t *fall_lambda = malloc(sizeof(uint64_t) * (size_t)(n + 1));
    int64_t *fin = malloc(sizeof(int64_t) * (size_t)N);
    int32_t *minmem = malloc(sizeof(int32_t) * (size_t)N);
    int32_t *rankof = malloc(sizeof(int32_t) * (size_t)N);
    int64_t *clist = malloc(sizeof(int64_t) * (size_t)N);
    if (!exists || !parent || !nsize || !coff || !kids || !node_cl || !stack || !leafstack ||
        !cparent || !cbirth || !cdeath || !csize || !sel || !stab || !S || !childsum ||
        !fall_cluster || !fall_lambda || !fin || !minmem || !rankof || !clist)
        return ORC_ERR_OOM;
#define LEVEL_NODE(i, c) ((int64_t)((i) + 1) * n + (c))
    /* the nodes of D and their parents */
    for (int64_t X = 0; X < N; X++) parent[X] = -1;
    exists[root] = 1;
    for (int64_t x = 0; x < n; x++) {
        exists[x] = 1;
        parent[x] = LEVEL_NODE(0, lab[x]);
    }
    for (int32_t i = 0; i < q; i++)
        for (int64_t c = 0; c < n; c++) {
            if (lab[(int64_t)i * n + c] != (int32_t)c) continue;
            int64_t X = LEVEL_NODE(i, c);
            exists[X] = 1;
            parent[X] = (i + 1 < q) ? LEVEL_NODE(i + 1, lab[(int64_t)(i + 1) * n + c]) : root;
        }
    /* sizes: members of each component */
    for (int64_t x = 0; x < n; x++) {
        nsize[x] = 1;
        for (int32_t i = 0; i < q; i++) nsize[LEVEL_NODE(i, lab[(int64_t)i * n + x])]++;
    }
    nsize[root] = n;
    /* children lists */
    for (int64_t X = 0; X < N; X++)
        if (exists[X] && parent[X] >= 0) coff[parent[X] + 1]++;
    for (int64_t X = 0; X < N; X++) coff[X + 1] += coff[X];
    {
        int64_t *f = malloc(sizeof(int64_t) * (size_t)N);
        if (!f) return ORC_ERR_OOM;
        memcpy(f, coff, sizeof(int64_t) * (size_t)N);
        for (int64_t X = 0; X < N; X++)
            if (exists[X] && parent[X] >= 0) kids[f[parent[X]]++] = X;
        free(f);
    }
#define NODE_LAMBDA(X) ((X) == root ? 0u : lam(omega[(X) / n - 1]))
    /* top-down walk from the root cluster */
    for (int64_t X = 0; X < N; X++) node_cl[X] = -1;
    node_cl[root] = root;
    cparent[root] = -1; cbirth[root] = 0; csize[root] = n;
    int64_t sp = 0;
    stack[sp++] = root;
    while (sp > 0) {
        int64_t X = stack[--sp];
        int64_t K = node_cl[X];
        uint64_t LX = NODE_LAMBDA(X);
        int64_t nbig = 0;
        for (int64_t y = coff[X]; y < coff[X + 1]; y++)
            if (nsize[kids[y]] >= M) nbig++;
        if (nbig >= 2) cdeath[K] = LX;
        for (int64_t y = coff[X]; y < coff[X + 1]; y++) {
            int64_t C = kids[y];
            if (nsize[C] >= M) {
                if (nbig >= 2) {
                    node_cl[C] = C;
                    cparent[C] = K; cbirth[C] = LX; csize[C] = nsize[C];
                } else {
                    node_cl[C] = K;
                }
                stack[sp++] = C;
            } else {
                int64_t lp = 0;
                leafstack[lp++] = C;
                while (lp > 0) {
                    int64_t Z = leafstack[--lp];
                    if (Z < n) { fall_cluster[Z] = K; fall_lambda[Z] = LX; }
                    else for (int64_t t = coff[Z]; t < coff[Z + 1]; t++) leafstack[lp++] = kids[t];
                }
            }
        }
    }
    /* stabilities */
    for (int64_t x = 0; x < n; x++)
        stab[fall_cluster[x]] += (u128)(fall_lambda[x] - cbirth[fall_cluster[x]]);
    int64_t ncl = 0;
    for (int64_t X = 0; X < N; X++)
        if (node_cl[X] == X) clist[ncl++] = X;          /* ascending: children first */
    for (int64_t c = 0; c < ncl; c++) {
        int64_t K = clist[c];
        if (cparent[K] >= 0)
            stab[cparent[K]] += (u128)csize[K] * (u128)(cdeath[cparent[K]] - cbirth[cparent[K]]);
    }
    /* excess of mass, bottom-up */
    for (int64_t c = 0; c < ncl; c++) {
        int64_t K = clist[c];
        if (K == root) continue;
        if (stab[K] >= childsum[K]) { sel[K] = 1; S[K] = stab[K]; }
        else { sel[K] = 0; S[K] = childsum[K]; }
        childsum[cparent[K]] += S[K];
    }
    /* final clusters: selected with no selected ancestor below the root */
    for (int64_t c = ncl - 1; c >= 0; c--) {
        int64_t K = clist[c];
        if (K == root) { fin[K] = -1; continue; }
        int64_t up = fin[cparent[K]];
        if (up >= 0) fin[K] = up;
        else if (sel[K]) { sel[K] = 2; fin[K] = K; }
        else fin[K] = -1;
    }
    for (int64_t X = 0; X < N; X++) { minmem[X] = INT32_MAX; rankof[X] = -1; }
    for (int64_t x = 0; x < n; x++) {
        int64_t L = fin[fall_cluster[x]];
        if (L >= 0 && (int32_t)x < minmem[L]) minmem[L] = (int32_t)x;
    }
    int32_t nlab = 0;
    for (int64_t x = 0; x < n; x++) {
        int64_t L = fin[fall_cluster[x]];
        if (L >= 0 && minmem[L] == (int32_t)x) rankof[L] = nlab++;
    }
    for (int64_t x = 0; x < n; x++) {
        int64_t L = fin[fall_cluster[x]];
        labels[x] = L >= 0 ? rankof[L] : -1;
    }
    for (int64_t c = 0; c < ncl; c++) {
        int64_t K = clist[c];
        cl_birth[c] = cbirth[K];
        cl_death[c] = cdeath[K];
        cl_size[c] = csize[K];
        cl_stab_hi[c] = (uint64_t)(stab[K] >> 64);
        cl_stab_lo[c] = (uint64_t)stab[K];
        cl_selected[c] = (K == root) ? 0 : sel[K];
    }
    *n_cl = ncl;
    *n_labels = nlab;
    free(exists); free(parent); free(nsize); free(coff); free(kids); free(node_cl);
    free(stack); free(leafstack); free(cparent); free(cbirth); free(cdeath); free(csize);
    free(sel); free(stab); free(S); free(childsum); free(fall_cluster); free(fall_lambda);
    free(fin); free(minmem); free(rankof); free(clist);
    return ORC_OK;
#undef LEVEL_NODE
#undef NODE_LAMBDA
}

/* ------------------------------------------------------------------ */
/* Dynamic hypergraphs (Sec. 4.4). Hyperedge r = (S_r, t_r) with its    */
/* members as CSR rows: s_off[E + 1], s_vert[s_off[E]]. The line graph */
/* joins two hyperedges that share a vertex, weight |t_r - t_s|.       */
/* Undirected: at every vertex the clique of incident hyperedges has   */
/* the time-sorted path as a local MST (ties by id). Directed: r also  */
/* has targets R_r (d_off, d_vert); at a vertex i the in-list holds the */
/* hyperedges with i in R (arriving) and the out-list those with i in  */
/* S (leaving), and Alg. 2 runs on them as for a graph. The skeleton   */
/* is the union over vertices as a set (u < v), sorted by (w, u, v).   */
/* Returns the link count, or -(error code). Capacity: s_off[E] +      */
/* d_off[E] links. Reading: a vertex listed twice in one member set, or */
/* (directed) in both S_r and R_r, is rejected like a self loop.       */
/* ------------------------------------------------------------------ */

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int hyper_check(int64_t E, int32_t V, const int64_t *off, const int32_t *vert,
                       int32_t *tmp)
{
    for (int64_t e = 0; e < E; e++) {
        int64_t n = off[e + 1] - off[e];
        if (n < 0) return ORC_ERR_ARG;
        for (int64_t x = 0; x < n; x++) {
            int32_t a = vert[off[e] + x];
            if (a < 0 || a >= V) return ORC_ERR_VERTEX;
            tmp[x] = a;
        }
        qsort(tmp, (size_t)n, sizeof(int32_t), cmp_i32);
        for (int64_t x = 1; x < n; x++)
            if (tmp[x] == tmp[x - 1]) return ORC_ERR_SELF_LOOP;
    }
    return ORC_OK;
}

int64_t orc_hyper_skeleton(int64_t E, int32_t V, const int64_t *t, int32_t directed,
                           const int64_t *s_off, const int32_t *s_vert,
                           const int64_t *d_off, const int32_t *d_vert,
                           int32_t *u_out, int32_t *v_out, int64_t *w_out)
{
    if (E < 0 || V < 0 || s_off[0] != 0 || (directed && d_off[0] != 0)) return -ORC_ERR_ARG;
    int64_t Ms = s_off[E], Md = directed ? d_off[E] : 0;
    int64_t cap = Ms + Md + 1;
    int32_t *tmp = malloc(sizeof(int32_t) * (size_t)cap);
    int64_t *deg = calloc((size_t)V + 1, sizeof(int64_t));
    inc_rec *all = malloc(sizeof(inc_rec) * (size_t)cap);
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)V + 1));
    int32_t *W = malloc(sizeof(int32_t) * (size_t)cap);
    wedge *links = malloc(sizeof(wedge) * (size_t)cap);
    if (!tmp || !deg || !all || !fill || !W || !links) return -ORC_ERR_OOM;
    int rc = hyper_check(E, V, s_off, s_vert, tmp);
    if (!rc && directed) rc = hyper_check(E, V, d_off, d_vert, tmp);
    if (!rc && directed) {                              /* no vertex in both S_r and R_r */
        for (int64_t e = 0; e < E && !rc; e++) {
            int64_t ns = s_off[e + 1] - s_off[e], nd = d_off[e + 1] - d_off[e];
            for (int64_t x = 0; x < ns && !rc; x++)
                for (int64_t y = 0; y < nd; y++)
                    if (s_vert[s_off[e] + x] == d_vert[d_off[e] + y]) { rc = ORC_ERR_SELF_LOOP; break; }
        }
    }
    if (rc) { free(tmp); free(deg); free(all); free(fill); free(W); free(links); return -rc; }
    /* incidence records per vertex: dir 1 = the vertex is in S (leaving),
     * dir 0 = in R (arriving); undirected members are all dir 1 */
    for (int64_t m = 0; m < Ms; m++) deg[s_vert[m] + 1]++;
    for (int64_t m = 0; m < Md; m++) deg[d_vert[m] + 1]++;
    for (int32_t i = 0; i < V; i++) deg[i + 1] += deg[i];
    memcpy(fill, deg, sizeof(int64_t) * ((size_t)V + 1));
    for (int64_t e = 0; e < E; e++) {
        inc_rec r;
        r.t = t[e]; r.id = (int32_t)e;
        r.dir = 1;
        for (int64_t m = s_off[e]; m < s_off[e + 1]; m++) all[fill[s_vert[m]]++] = r;
        r.dir = 0;
        if (directed)
            for (int64_t m = d_off[e]; m < d_off[e + 1]; m++) all[fill[d_vert[m]]++] = r;
    }
    int64_t n = 0;
    for (int32_t i = 0; i < V; i++) {
        inc_rec *Ei = all + deg[i];
        int64_t di = deg[i + 1] - deg[i];
        qsort(Ei, (size_t)di, sizeof(inc_rec), cmp_inc);   /* sort by time, ties by id */
        if (!directed) {
            for (int64_t x = 1; x < di; x++) {              /* the path through E_i */
                int32_t a = Ei[x - 1].id, b = Ei[x].id;
                links[n].u = a < b ? a : b;
                links[n].v = a < b ? b : a;
                links[n].w = Ei[x].t - Ei[x - 1].t;
                n++;
            }
        } else {
            int64_t wlen = 0;                               /* Alg. 2 with W */
            for (int64_t x = 0; x < di; x++) {
                if (Ei[x].dir == 0) {
                    W[wlen++] = Ei[x].id;
                } else {
                    for (int64_t y = 0; y < wlen; y++) {
                        int32_t a = W[y], b = Ei[x].id;
                        links[n].u = a < b ? a : b;
                        links[n].v = a < b ? b : a;
                        links[n].w = Ei[x].t - t[W[y]];
                        n++;
                    }
                    if (wlen > 0) { W[0] = W[wlen - 1]; wlen = 1; }
                }
            }
        }
    }
    qsort(links, (size_t)n, sizeof(wedge), cmp_wedge);     /* the union, as a set */
    int64_t m = 0;
    for (int64_t x = 0; x < n; x++) {
        if (m > 0 && cmp_wedge(&links[m - 1], &links[x]) == 0) continue;
        links[m++] = links[x];
    }
    for (int64_t x = 0; x < m; x++) { u_out[x] = links[x].u; v_out[x] = links[x].v; w_out[x] = links[x].w; }
    free(tmp); free(deg); free(all); free(fill); free(W); free(links);
    return m;
}
