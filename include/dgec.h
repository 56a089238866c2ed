/*
 * dgec.h -- C ABI of the GB300 (sm_103a) implementation of the edge
 * clustering method of "Scalable Edge Clustering of Dynamic Graphs via
 * Weighted Line Graphs" (arXiv 2311.10337).
 *
 * The problem (Sec. 1.2.1, Alg. 4): a dynamic multigraph is a list of
 * directed temporal edges e = (i_e, j_e, t_e); no self loops; no two edges
 * share (i, j, t). Each edge is a node of the increment-weighted line graph
 * L_G (Def. 1): arc r -> s iff j_r == i_s and t_r <= t_s, weight t_s - t_r.
 * The library clusters the edges by running hierarchical agglomerative
 * clustering (Alg. 1) on the line-graph skeleton L*_G (Alg. 2-3), which has
 * the same weighted connectivity as L_G (Thm. 3) but at most 2|E| - |V|
 * edges, so L_G is never formed.
 *
 * Conventions for every call:
 *   - an edge's id is its position in the input arrays (0 .. n_edges-1);
 *     ids are the line-graph nodes and the final tie-break everywhere;
 *   - pointers named d_* are device pointers, h_* host pointers; the caller
 *     owns all input memory and the workspace; the library never frees it;
 *   - the library reads inputs and never writes them;
 *   - all arithmetic is integer, so results are exact and reproducible;
 *   - every call runs on the given CUDA stream and returns once its results
 *     are complete (it synchronises that stream before returning);
 *   - on error the call returns a status != DGEC_OK and a message is kept in
 *     the context (dgec_last_error); outputs are then unspecified;
 *   - a context serves one call at a time (it holds that call's stream,
 *     message, launch count and timers): threads that share one must
 *     serialise their calls, or each use its own context, as the server's
 *     lanes do. The size queries and dgec_status_string are safe from any
 *     thread; the server calls and dgec_msf_static state their own rules.
 */
#ifndef DGEC_H
#define DGEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DGEC_OK = 0,
    DGEC_ERR_INVALID_ARG = 1,   /* null pointer, negative size, k or M out of range */
    DGEC_ERR_VERTEX_RANGE = 2,  /* a src/dst outside [0, n_vertices) */
    DGEC_ERR_SELF_LOOP = 3,     /* an edge (i, i, t): excluded by Sec. 1.2.1 */
    DGEC_ERR_TOO_LARGE = 4,     /* n_edges >= 2^30, or time span too wide (see below) */
    DGEC_ERR_OOM = 5,           /* workspace smaller than dgec_workspace_size() */
    DGEC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    DGEC_ERR_TIMEOUT = 7,       /* an iterative stage exceeded its round bound, or a wait timed out */
    DGEC_ERR_ADMISSION = 8,     /* a served job can never fit a lane's memory */
    DGEC_ERR_INTERNAL = 9
} dgec_status;

/* flags of dgec_params */
#define DGEC_CUTOFF 1u  /* time cutoff of Sec. 4.3: keep only line-graph arcs with w <= delta_max */
/* Mutual-reachability mode -- an approximation with no counterpart in the
 * paper: cluster the graph H = L*_G together with every edge's kNN pairs
 * (each pair once), weighed max(core_a, core_b, |t_a - t_b|) as in HDBSCAN,
 * instead of L*_G under P3. Pairs with an endpoint of infinite core (fewer
 * than k neighbours) are dropped. Thm. 3 does not hold for these weights, so
 * H does not reproduce clustering the full line graph with them; with k = 1
 * the result equals the plain method. The skeleton outputs stay L*_G; the
 * forest, dendrogram, condensed tree and labels refer to H. Uses about
 * (2 + k) * 40 more workspace bytes per edge. */
#define DGEC_MRD 2u
/* Nearly-causal line graph of Sec. 4.3: an arc r -> s (dst r = src s) also
 * exists when s is at most delta_nc earlier than r (t_s >= t_r - delta_nc),
 * weighed |t_s - t_r|, to absorb timestamp error. Its skeleton is L*_G
 * together with the links of the skeleton of G with negated times whose
 * weight is <= delta_nc (an MST of a union of graphs lies in the union of
 * their MSTs; on negated times Alg. 2 gives the backward arcs' MST), which
 * keeps the weighted connectivity; the kNN lists count backward neighbours
 * within delta_nc too. The skeleton outputs are then ordered by (u, v).
 * delta_nc = 0 is the causal method. Not combined with DGEC_MRD. */
#define DGEC_NEARLY_CAUSAL 4u

typedef struct {
    int32_t k;                /* neighbours per edge for the kNN output, 1 <= k <= 16 */
    int32_t min_cluster_size; /* M of Alg. 1's condensing, M >= 2 */
    uint32_t flags;           /* 0, or any of DGEC_CUTOFF, DGEC_MRD, DGEC_NEARLY_CAUSAL */
    int64_t delta_max;        /* with DGEC_CUTOFF: the cutoff, >= 0 (ignored otherwise). Only arcs
                                 with w <= delta_max are in the line graph: the skeleton keeps the
                                 links with w <= delta_max (exact by Thm. 3), the kNN lists only
                                 neighbours within delta_max, and everything downstream follows. */
    int64_t delta_nc;         /* with DGEC_NEARLY_CAUSAL: the tolerance, >= 0 (ignored otherwise) */
} dgec_params;

typedef struct dgec_ctx dgec_ctx;

/* Results of dgec_run. Device arrays point into the caller's workspace and
 * stay valid until that workspace is reused. Counts are host values. */
typedef struct {
    /* Incidence lists (the adjacency lists Alg. 3 starts from). Vertex v's
     * out-edges are out_id[out_off[v] .. out_off[v+1]) with times
     * out_t[..], sorted by (t, id); likewise in-edges via in_off/in_t/in_id. */
    const int64_t *out_off, *in_off;   /* [n_vertices + 1] */
    const int64_t *out_t, *in_t;       /* [n_edges] */
    const int32_t *out_id, *in_id;     /* [n_edges] */
    /* Each edge's place in those arrays: out_id[pos_out[e]] == e and
     * in_id[pos_in[e]] == e; its index within src's list is
     * pos_out[e] - out_off[src[e]] (likewise for dst's in-list). */
    const int32_t *pos_out, *pos_in;   /* [n_edges] */
    /* Alg. 3: skeleton L*_G as undirected edges (u < v, w = |t_u - t_v|),
     * each line-graph edge once. Deterministic order (not sorted by (w, u,
     * v): the forest below is): first every edge's link to the first later
     * out-edge at its head, in the order of the in-lists (by head vertex,
     * then (t, id)); then every edge's link to the retained in-edge at its
     * tail, in the order of the out-lists (by tail vertex, then (t, id)). */
    const int32_t *sk_u, *sk_v;        /* [n_skeleton] */
    const int64_t *sk_w;
    /* k nearest line-graph neighbours in time: knn_id[e*k + x], ranked by
     * (|dt|, id), -1 padded; core[e] = |dt| of the k-th, INT64_MAX if the
     * node has fewer than k neighbours. */
    const int32_t *knn_id;             /* [n_edges * k] */
    const int64_t *core;               /* [n_edges] */
    /* Alg. 1, forest and its weight order: minimum spanning forest of L*_G
     * under the strict order (w, u, v), sorted by that order. */
    const int32_t *mst_u, *mst_v;      /* [n_mst] */
    const int64_t *mst_w;
    /* Alg. 1, union-find dendrogram. Row s merges clusters link_a[s] <
     * link_b[s] (a leaf id < n_edges, or n_edges + s' for the cluster row s'
     * formed) at weight mst_w[s]; link_size[s] leaves below it. */
    const int32_t *link_a, *link_b;    /* [n_mst] */
    const int64_t *link_size;
    /* Alg. 1, condensing and cluster extraction: condensed tree (min cluster
     * size M) and excess of mass selection. lambda(w) = floor((2^64-1)/(w+1)); lambda 0 at a
     * virtual root (id n_edges + n_mst) above the components. Point e
     * leaves cluster fall_cluster[e] at lambda fall_lambda[e]. Clusters,
     * sorted by id (the dendrogram node where each is born): parent id
     * (-1 for the root), birth and death lambda (death 0 if it never
     * splits), size at birth, stability as a 128-bit integer (hi, lo),
     * selected = 2 final, 1 selected but inside a selected ancestor, 0 no. */
    const int32_t *fall_cluster;       /* [n_edges] */
    const uint64_t *fall_lambda;       /* [n_edges] */
    const int32_t *cl_id, *cl_parent;  /* [n_condensed] */
    const uint64_t *cl_birth, *cl_death, *cl_stab_hi, *cl_stab_lo;
    const int64_t *cl_size;
    const int32_t *cl_selected;
    /* Alg. 4 output: edge clusters; -1 = noise; clusters numbered
     * 0 .. n_clusters-1 by their smallest member id. */
    const int32_t *labels;             /* [n_edges] */
    int64_t n_skeleton, n_mst, n_condensed;
    int32_t n_clusters;
} dgec_result;

/* Context bound to one CUDA device. Owns only host memory and a small
 * pinned buffer; never allocates device memory. */
dgec_status dgec_create(dgec_ctx **out, int device);
dgec_status dgec_destroy(dgec_ctx *ctx);
/* Message of the last failed call on ctx ("" if none). */
const char *dgec_last_error(const dgec_ctx *ctx);
const char *dgec_status_string(dgec_status s);

/* Bytes of device workspace dgec_run needs for these sizes. The bound is
 * independent of the edge values. n_edges < 2^30, n_vertices >= 0. */
dgec_status dgec_workspace_size(int64_t n_edges, int32_t n_vertices,
                                const dgec_params *params, size_t *bytes);

/*
 * Alg. 4 end to end on device-resident edges: incidence lists (the
 * adjacency lists Alg. 3 starts from), skeleton (Alg. 2-3), kNN and core distances, minimum
 * spanning forest, dendrogram, condensed tree, labels (Alg. 1).
 * d_src, d_dst: int32[n_edges] vertex ids in [0, n_vertices);
 * d_t: int64[n_edges] times. The time span (max t - min t) must satisfy
 * bits(span) + bits(n_edges - 1) <= 64. d_workspace: >= ws_bytes bytes,
 * 256-byte aligned, from dgec_workspace_size. Fills *out.
 */
dgec_status dgec_run(dgec_ctx *ctx, const int32_t *d_src, const int32_t *d_dst,
                     const int64_t *d_t, int64_t n_edges, int32_t n_vertices,
                     const dgec_params *params, void *d_workspace,
                     size_t ws_bytes, void *cuda_stream, dgec_result *out);

/*
 * Same computation from host memory: copies h_src/h_dst/h_t (pinned memory
 * makes the copies asynchronous) into the workspace, runs dgec_run, and
 * copies the labels back to h_labels (int32[n_edges]). The workspace must
 * hold dgec_workspace_size() + 16 * n_edges + 1024 bytes.
 */
dgec_status dgec_run_host(dgec_ctx *ctx, const int32_t *h_src,
                          const int32_t *h_dst, const int64_t *h_t,
                          int64_t n_edges, int32_t n_vertices,
                          const dgec_params *params, void *d_workspace,
                          size_t ws_bytes, void *cuda_stream,
                          int32_t *h_labels, int32_t *h_n_clusters);

/*
 * Batched form: many independent graphs in one pass of the pipeline (the
 * paper has no batched form; its method per graph is unchanged, Alg. 4
 * runs on each graph as if alone). Graph g owns the
 * input edges [h_edge_off[g], h_edge_off[g+1]) of d_src/d_dst/d_t, with
 * vertex ids local to the graph in [0, h_n_vertices[g]), its own k and
 * min cluster size, and its own virtual root. Every result equals the
 * result of dgec_run on that graph alone.
 */
typedef struct {
    /* per-edge outputs, graph after graph, in each graph's local ids */
    const int32_t *labels;     /* [total_edges]: -1 noise, else 0..n_clusters[g]-1 */
    const int32_t *knn_id;     /* graph g's rows start at knn_off[g]; k_g local ids per edge */
    const int64_t *core;       /* [total_edges] */
    /* forest and dendrogram rows of graph g: [mst_off[g], mst_off[g+1]),
     * (w, u, v) order, local ids; a dendrogram child >= E_g is E_g + the
     * local row that formed it */
    const int32_t *mst_u, *mst_v;
    const int64_t *mst_w;
    const int32_t *link_a, *link_b;
    const int64_t *link_size;
    /* per-graph device tables */
    const int32_t *n_clusters;  /* [n_graphs] */
    const int64_t *mst_off;     /* [n_graphs + 1] */
    const int64_t *knn_off;     /* [n_graphs + 1] */
    int64_t total_edges, total_mst;
    int32_t total_clusters;
    /* the whole batch as one dgec_result in global ids (edge id = position
     * in the batch, vertex id = local id + the vertex counts of earlier
     * graphs); its condensed-tree arrays carry one virtual root per graph */
    dgec_result global;
} dgec_batch_result;

/* Workspace bytes for a batch; the tables are host arrays. */
dgec_status dgec_batch_workspace_size(int32_t n_graphs, const int64_t *h_edge_off,
                                      const int32_t *h_n_vertices, const int32_t *h_k,
                                      const int32_t *h_min_cluster_size, size_t *bytes);
/* Runs the batch; h_edge_off[0] must be 0; limits and errors as dgec_run
 * (total edges < 2^30, total vertices < 2^31). */
dgec_status dgec_run_batch(dgec_ctx *ctx, int32_t n_graphs, const int64_t *h_edge_off,
                           const int32_t *h_n_vertices, const int32_t *h_k,
                           const int32_t *h_min_cluster_size, const int32_t *d_src,
                           const int32_t *d_dst, const int64_t *d_t, void *d_workspace,
                           size_t ws_bytes, void *cuda_stream, dgec_batch_result *out);

/*
 * Serving: a request loop with continuous batching of windowed clustering
 * jobs (no counterpart in the paper). The server splits a caller-provided
 * device pool into n_lanes lanes, each with its own host thread, CUDA
 * stream and workspace.
 * A free lane takes, in arrival order, every pending job that fits its
 * memory (admission by memory), renumbers each job's vertices densely on
 * the device, runs them together as one batch (dgec_run_batch) and writes
 * each job's labels. Jobs that arrive while lanes are busy are picked up by
 * the next lane to free up, so their work overlaps on the device. A job's
 * result is identical whether it runs alone or in a mix.
 */
typedef struct dgec_server dgec_server;

typedef struct {
    const int32_t *d_src, *d_dst;  /* device, caller-owned, read during the job */
    const int64_t *d_t;
    int64_t n_edges;
    int32_t k;                     /* 1..16 */
    int32_t min_cluster_size;      /* >= 2 */
    int32_t *d_labels;             /* device, caller-owned, int32[n_edges] output */
} dgec_job;

/* pool: device memory owned by the caller for the server's lifetime; it is
 * split into n_lanes equal lanes. Vertex ids of every job must lie in
 * [0, vertex_bound). max_jobs_per_batch caps a lane's batch. */
dgec_status dgec_server_create(int device, void *d_pool, size_t pool_bytes, int32_t n_lanes,
                               int32_t vertex_bound, int32_t max_jobs_per_batch,
                               dgec_server **out);
/* Queue a job (thread-safe, returns at once). *ticket names it in dgec_wait. */
dgec_status dgec_submit(dgec_server *srv, const dgec_job *job, uint64_t *ticket);
/* Wait for a job (timeout_ms < 0: no limit). On success fills the number of
 * clusters and the job's latency from submission to labels ready (ms).
 * Returns the job's own status (e.g. DGEC_ERR_SELF_LOOP for a bad job,
 * DGEC_ERR_ADMISSION if it can never fit a lane). A ticket can be waited
 * for once. */
dgec_status dgec_wait(dgec_server *srv, uint64_t ticket, int32_t timeout_ms,
                      int32_t *n_clusters, double *latency_ms);
/* Edge capacity of one lane (the largest job it can admit). */
int64_t dgec_server_lane_capacity(const dgec_server *srv);
/* Stops the lanes after the jobs already taken and frees host state; the
 * pool is untouched. Jobs still queued complete with DGEC_ERR_INVALID_ARG. */
dgec_status dgec_server_destroy(dgec_server *srv);

/* Launch configuration of the calls made on ctx (no counterpart in the
 * paper; it changes speed, never results): threads per CTA of the kNN kernel
 * (64, 128 or 256; default 128), the number of CTAs of each grid-stride
 * streaming kernel (1 .. 2^20; default 65,536), and the form of the kNN
 * kernel (knn_packed): 0 reads separate time and id arrays; 1 reads its
 * windows from packed 64-bit list keys ((t - tmin) << 32 | id) and sorts its
 * candidates as packed keys (|dt| << 32 | id), one edge a thread; 2 (the
 * default) does the same in list order, one pass over the out-lists for the
 * predecessor windows and one over the in-lists for the successor windows,
 * with K keys an edge held in the workspace in between. Forms 1 and 2 apply
 * only when the time span fits 32 bits (else form 0 runs). The autotuner of
 * the Python package picks them per GPU model and workload. Invalid values
 * give DGEC_ERR_INVALID_ARG and leave the configuration unchanged. */
typedef struct {
    int32_t knn_block;
    int32_t stream_ctas;
    int32_t knn_packed;
} dgec_launch_config;
dgec_status dgec_set_launch_config(dgec_ctx *ctx, const dgec_launch_config *cfg);
dgec_status dgec_get_launch_config(const dgec_ctx *ctx, dgec_launch_config *cfg);

/* Device time of each pipeline stage of the last completed call on ctx
 * (dgec_run, dgec_run_host, dgec_run_batch, dgec_run_levels,
 * dgec_run_hyper), from CUDA events recorded on the call's stream at the
 * stage boundaries: the i-th stage's name (static string, e.g. "A incidence
 * lists", "B skeleton and kNN", "C spanning forest", "D1 dendrogram",
 * "D2 condense and labels") and its milliseconds. Returns
 * DGEC_ERR_INVALID_ARG when i is past the last stage. */
dgec_status dgec_stage_timing(const dgec_ctx *ctx, int i, const char **name, double *ms);

/* Number of kernel launches the last dgec_run on ctx issued (for reporting). */
int64_t dgec_last_launch_count(const dgec_ctx *ctx);

/* Measurement aid: time kernels with CUDA events recorded on the run's
 * stream around each launch. mode 0 = off, 1 = only launches of the kernel
 * called `name` (e.g. "k_knn"), 2 = every launch, 3 = launches of every
 * kernel whose name starts with `name` (e.g. "k_knn": the kNN step in any
 * form, one launch or the two passes "k_knn_pred" and "k_knn"). Resets the
 * totals. */
dgec_status dgec_set_kernel_timing(dgec_ctx *ctx, int mode, const char *name);
/* Totals since the last reset for the i-th kernel name seen (0-based):
 * its name (static string), summed milliseconds and launch count.
 * Returns DGEC_ERR_INVALID_ARG when i is past the last name. */
dgec_status dgec_kernel_timing(dgec_ctx *ctx, int i, const char **name, double *total_ms,
                               int64_t *launches);

/*
 * Minimum spanning forest without any device allocation. The paper has no
 * counterpart to this call: it exists for callers that may not allocate
 * device memory where they need a forest (a plugin inside a framework that
 * owns all device memory, a loop that forbids allocation after start-up, a
 * thread that cannot reach cudaMalloc). Its working memory is one fixed
 * array of about 22 MB that the library reserves on every device it is
 * loaded onto, for the life of the process.
 *
 * Input: d_u, d_v, d_w: n_edges undirected edges over nodes 0..n_nodes-1,
 * each written with d_u < d_v (as dgec_result's skeleton is), w >= 0.
 * Output: the minimum spanning forest under the strict order (w, u, v) --
 * the same edge set dgec_run returns in mst_u/mst_v/mst_w -- written in no
 * particular order to d_mst_u/d_mst_v/d_mst_w (capacity n_nodes - 1), its
 * size to *h_n_mst. Runs on cuda_stream of the current device and
 * synchronises it before returning.
 * Limits: n_nodes <= 262,144 and n_edges <= 524,288, else
 * DGEC_ERR_TOO_LARGE; a bad id, u >= v or w < 0 gives
 * DGEC_ERR_INVALID_ARG (nothing is written to the outputs then).
 * It synchronises the stream once per Boruvka round (a counter read), so it
 * cannot be stream-captured. Every call reuses the same array (each call
 * re-initialises what must start from a known value), so calls that
 * overlap on the GPU race with each other: serialise them.
 */
dgec_status dgec_msf_static(const int32_t *d_u, const int32_t *d_v, const int64_t *d_w,
                            int64_t n_edges, int64_t n_nodes, int32_t *d_mst_u,
                            int32_t *d_mst_v, int64_t *d_mst_w, int64_t *h_n_mst,
                            void *cuda_stream);

/* ---------------------------------------------------------------------
 * Discrete dendrogram (Alg. 5, Sec. 3).
 *
 * Given thresholds omega_0 < omega_1 < ... < omega_{q-1}, level i is the
 * partition comps(L*_G, omega_i) of the edges: two edges share a component
 * when a path of skeleton links of weight <= omega_i joins them (Alg. 5
 * admits links strictly below the threshold, the appendix links up to it;
 * the latter is used, so a threshold equal to a weight admits it). By Thm. 3 these are the components of L_G itself.
 * Components are named by their smallest member edge id; levels are nested
 * and D is the tree of containments between consecutive levels.
 *
 * D in per-edge form: edge x names its component at every level below
 * merge_level[x]; at level merge_level[x] its component becomes part of the
 * component named merge_parent[x] (< x). Both are -1 for an edge that names
 * its component at every level. The label of x at level i is found by
 * following merge_parent while merge_level <= i.
 *
 * With min_cluster_size M >= 2, the HDBSCAN condensed tree is built on D
 * (Sec. 3, condensing on the discrete dendrogram): every event of level i
 * happens at lambda(omega_i) = floor((2^64 - 1) / (omega_i + 1)), a
 * virtual root at lambda 0 joins the last level's components, and the
 * excess-of-mass selection and labels follow the conventions of dgec_run
 * (-1 noise, clusters numbered by smallest member, root never selected).
 * --------------------------------------------------------------------- */
#define DGEC_MAX_LEVELS 64
#define DGEC_LEVELS_DENSE 1u  /* also write every level's labels */

typedef struct {
    int32_t n_levels;          /* q, 1 <= q <= DGEC_MAX_LEVELS */
    const int64_t *h_omega;    /* host int64[q], 0 <= omega_0 < omega_1 < ... */
    int32_t min_cluster_size;  /* 0: no condensing; else M >= 2 */
    uint32_t flags;            /* 0 or DGEC_LEVELS_DENSE */
} dgec_levels_params;

/* Results of dgec_run_levels: device arrays in the caller's workspace,
 * valid until it is reused; counts are host values. */
typedef struct {
    const int32_t *sk_u, *sk_v;       /* skeleton, as in dgec_result */
    const int64_t *sk_w;
    const int32_t *merge_level;       /* [n_edges] */
    const int32_t *merge_parent;      /* [n_edges] */
    const int64_t *n_components;      /* [q] components at each level */
    const int32_t *level_labels;      /* [q * n_edges], row i = level i; NULL without DGEC_LEVELS_DENSE */
    const int32_t *labels;            /* [n_edges] condensed labels; NULL when M == 0 */
    int64_t n_skeleton;
    int64_t n_merges;                 /* edges of D = n_edges - components at the last level */
    int32_t n_clusters;
} dgec_levels_result;

/* Bytes of device workspace dgec_run_levels needs. */
dgec_status dgec_levels_workspace_size(int64_t n_edges, int32_t n_vertices,
                                       const dgec_levels_params *params, size_t *bytes);

/*
 * Incidence lists, skeleton (Alg. 2-3), the discrete dendrogram D (Alg. 5)
 * and, when M >= 2, its condensed labels, on device-resident edges (same
 * input rules as dgec_run; no kNN lists are computed). Thresholds that are
 * not strictly increasing, negative, or more than DGEC_MAX_LEVELS give
 * DGEC_ERR_INVALID_ARG. Fills *out.
 */
dgec_status dgec_run_levels(dgec_ctx *ctx, const int32_t *d_src, const int32_t *d_dst,
                            const int64_t *d_t, int64_t n_edges, int32_t n_vertices,
                            const dgec_levels_params *params, void *d_workspace,
                            size_t ws_bytes, void *cuda_stream, dgec_levels_result *out);

/* ---------------------------------------------------------------------
 * Dynamic hypergraphs (Sec. 4.4).
 *
 * A dynamic hyperedge e = (S_e, t_e) is a set of vertices observed at time
 * t_e; hyperedges are the nodes of the line graph, and two hyperedges that
 * share a vertex are joined with weight |t_r - t_s|. Directed hyperedges
 * have sources S_e and targets R_e; an arc r -> s exists when a target of r
 * is a source of s and t_r <= t_s (weight t_s - t_r), clustered by weak
 * connectivity as for graphs. The skeleton is the union over vertices of a
 * local MST (undirected: the path through the vertex's hyperedges in (t, id)
 * order; directed: Alg. 2 on the vertex's in-list R and out-list S), with
 * the same weighted connectivity as the line graph and at most
 * sum_i (d_i - 1) links; Alg. 1 then runs on it (forest, dendrogram,
 * condensed tree, labels; no kNN lists).
 *
 * Members are CSR rows: hyperedge e's sources (or members) are
 * d_src_vert[d_src_off[e] .. d_src_off[e+1]), its targets likewise in the
 * dst arrays (directed only; pass NULL and 0 otherwise). Offsets start at 0,
 * do not decrease and end at the member count. A vertex listed twice in one
 * member set, or in both S_e and R_e, gives DGEC_ERR_SELF_LOOP (the analogue
 * of Sec. 1.2.1's excluded self loops). Empty member sets are allowed.
 * --------------------------------------------------------------------- */
typedef struct {
    int32_t directed;          /* 0: undirected, 1: directed */
    int32_t min_cluster_size;  /* M >= 2 */
    uint32_t flags;            /* reserved, must be 0 */
} dgec_hyper_params;

/* Results of dgec_run_hyper: device arrays in the caller's workspace, valid
 * until it is reused; counts are host values. */
typedef struct {
    /* per vertex, the hyperedges having it as a member (directed: as a
     * source), in (t, id) order: src_list[src_voff[v] .. src_voff[v+1]) */
    const int64_t *src_voff;           /* [n_vertices + 1] */
    const int32_t *src_list;           /* [n_src_members] */
    const int64_t *dst_voff;           /* directed: as a target; NULL otherwise */
    const int32_t *dst_list;           /* [n_dst_members] */
    const int32_t *sk_u, *sk_v;        /* skeleton links u < v, w = |t_u - t_v|, [n_skeleton], */
    const int64_t *sk_w;               /* ordered by the (t, id) ranks of their two ends (earlier end first) */
    const int32_t *mst_u, *mst_v;      /* forest in (w, u, v) order, as in dgec_result */
    const int64_t *mst_w;
    const int32_t *link_a, *link_b;    /* dendrogram, as in dgec_result */
    const int64_t *link_size;
    const int32_t *labels;             /* [n_hyperedges], -1 noise */
    int64_t n_skeleton, n_mst;
    int32_t n_clusters;
} dgec_hyper_result;

dgec_status dgec_hyper_workspace_size(int64_t n_hyperedges, int32_t n_vertices,
                                      int64_t n_src_members, int64_t n_dst_members,
                                      const dgec_hyper_params *params, size_t *bytes);

dgec_status dgec_run_hyper(dgec_ctx *ctx, const int64_t *d_t, int64_t n_hyperedges,
                           int32_t n_vertices, const int64_t *d_src_off,
                           const int32_t *d_src_vert, int64_t n_src_members,
                           const int64_t *d_dst_off, const int32_t *d_dst_vert,
                           int64_t n_dst_members, const dgec_hyper_params *params,
                           void *d_workspace, size_t ws_bytes, void *cuda_stream,
                           dgec_hyper_result *out);

#ifdef __cplusplus
}
#endif
#endif /* DGEC_H */
