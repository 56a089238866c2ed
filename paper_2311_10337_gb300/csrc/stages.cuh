// Stage interfaces of the dgec pipeline (one translation unit per stage).
#pragma once

#include "prims.cuh"

namespace dgec {

// Problem description shared by the stages. A run is a batch of G >= 1
// independent graphs laid end to end (a plain run is G = 1): graph g owns
// edges [eoff[g], eoff[g+1]) with local vertex ids in [0, voff[g+1] -
// voff[g]); stages work on global ids (edge position, vertex + voff[g]).
struct Problem {
    const int32_t *src, *dst;
    const int64_t *t;
    int64_t E;
    int64_t V;  // total vertices
    int32_t k, M;  // largest k, smallest M over the graphs (host-side bounds)
    int64_t tmin = 0;
    int idbits = 1, tbits = 0;
    // per-graph description (device arrays)
    int32_t G = 1;
    const int64_t *eoff = nullptr;    // [G+1]
    const int64_t *voff = nullptr;    // [G+1]
    const int32_t *gk = nullptr;      // [G] k of each graph
    const int32_t *gM = nullptr;      // [G] M of each graph
    const int64_t *knn_off = nullptr; // [G+1] first kNN slot of each graph
    int32_t *egraph = nullptr;        // [E] graph of each edge (built in stage A)
    bool knn = true;                  // stage B also writes the kNN lists
    int knn_form = 0;                 // kNN kernel form, fixed in stage A (knn_packed, when the span allows)
    int64_t dmax = INT64_MAX;         // time cutoff (Sec. 4.3): only links with w <= dmax
    int64_t links_cap = -1;           // skeleton capacity; -1 = 2E (graphs: <= 2 links per edge)
    bool mrd = false;                 // cluster the mutual-reachability graph (stage M)
    int64_t dnc = 0;                  // nearly-causal tolerance (Sec. 4.3); 0 = causal (stage N off)
};

inline int64_t link_cap(const Problem &p) { return p.links_cap >= 0 ? p.links_cap : 2 * p.E; }

// Sorting u64 keys within per-vertex segments (off[V+1]) by the bin their
// length falls in (warp / CTA bitonic networks, hubs through the radix sort).
struct SegSort {
    int *bin_cnt, *bin_list;
    long long *scan_tmp, *hoff, *hsz;
    unsigned long long *hk, *hv, *hk2, *hv2;
    void *radix;
};
void carve_segsort(Arena &a, int64_t V, int64_t n, SegSort &s);
dgec_status sort_segments(Ctx *c, int64_t V, unsigned long long *keys, const int64_t *off, SegSort &s,
                          int key_bits);

// Stage A: incidence lists (Alg. 3's adjacency lists), per-vertex lists sorted by
// (t, id), and the merge ranks of Alg. 2 (from one sort of the merged lists).
//
// Internal numbering: every later stage names a line-graph node (a temporal
// edge) by r = its rank in (t, id) order. Skeleton links join edges that are
// close in time, so under r their two ends sit close in memory and the
// label/best-edge arrays of the forest and dendrogram stages are read with
// locality instead of at random. Original ids stay in every output and in
// every tie-break key.
struct Csr {
    int64_t *out_off, *in_off;  // [V+1]
    int64_t *out_t, *in_t;      // [E]
    int32_t *out_id, *in_id;    // [E] original ids (outputs)
    int32_t *out_r, *in_r;      // [E] internal ids of the same entries
    int32_t *orig_of;           // [E] r -> original id
    int32_t *rank_of;           // [E] original id -> r (read by the forest, levels, MRD and NC stages)
    int32_t *isrc, *idst;       // [E] src, dst in r order
    int64_t *it;                // [E] t in r order
    int4 *outrk;                // [E] by r: (.x) global slot in the out-lists, (.y) b = #in-edges of
                                //   src with t <= t_r, (.z) first slot of src's in-list (one record:
                                //   written together, read together)
    int2 *inrk;                 // [E] by r: (.x) first slot of dst's out-list not before t_r, (.y) end
                                //   of dst's out-list (a = .x - out_off[dst] = #out-edges with t < t_r)
    int32_t *pos_out, *pos_in;  // [E] by original id: position in out_id / in_id (outputs)
    int2 *in_va, *out_vb;       // [E] by list slot: (vertex, a) of each in-list entry, (vertex, b) of
                                //   each out-list entry (the skeleton pass walks the lists in order)
    int32_t *in_gs;             // [E] by in-list slot: first slot of its tie group (same vertex, same t)
    unsigned long long *out_key, *in_key;  // [E] by list slot, written when every t - tmin fits 32 bits:
                                           //   (t - tmin) << 32 | original id, so a kNN window is one run
                                           //   of one array
};
void plan_csr(Arena &ws, const Problem &p, Csr &o);
size_t csr_scratch_bytes(const Problem &p);
dgec_status stage_csr(Ctx *c, Problem &p, Csr &o, void *scratch);

// Stage B: skeleton (Alg. 2 as rank arithmetic + Alg. 3 union) and the
// k-nearest-in-time neighbours.
struct Skel {
    int32_t *u, *v;          // [2E] capacity; original ids, u < v (output)
    int32_t *ru, *rv;        // [2E] the same links in internal ids
    int64_t *w;
    int64_t n = 0;
    int32_t *knn;  // [E*k]
    int64_t *core;  // [E]
};
void plan_skel(Arena &ws, const Problem &p, Skel &o);
size_t skel_scratch_bytes(const Problem &p);
// also writes the kNN ids and core distances (same searches) unless p.knn is off
dgec_status stage_skeleton(Ctx *c, const Problem &p, const Csr &g, Skel &o, void *scratch);

// Stage M (optional): the mutual-reachability graph H = L* plus every kNN
// pair, weighed max(core_a, core_b, |dt|); an approximation (Thm. 3 does not
// hold for these weights). Capacity: link_cap(p) = 2E + E k.
void plan_mrd(Arena &ws, const Problem &p, Skel &h);
size_t mrd_scratch_bytes(const Problem &p);
dgec_status stage_mrd(Ctx *c, const Problem &p, const Csr &g, const Skel &sk, Skel &h, void *scratch);

// Stage N (optional): the nearly-causal line graph (Sec. 4.3). Stages A and
// B run again on the negated times (stage_nc_negate fills tn); stage_nc
// unites the two skeletons (backward links with w <= dnc) and merges the two
// kNN rows of every edge into h.knn / h.core. Capacity 4E links.
void plan_nc(Arena &ws, const Problem &p, Skel &h);
size_t nc_scratch_bytes(const Problem &p);
dgec_status stage_nc_negate(Ctx *c, const Problem &p, int64_t *tn);
dgec_status stage_nc(Ctx *c, const Problem &p, const Csr &g, const Skel &s1, const Skel &s2, Skel &h,
                     void *scratch);

// Stage C: minimum spanning forest of the skeleton (Borůvka), sorted by
// (w, u, v).
struct Msf {
    int32_t *u, *v;    // [E] original ids (output)
    int32_t *ru, *rv;  // [E] internal ids of the same edges
    int64_t *w;
    int64_t n = 0;
    int64_t *goff;     // [G+1] rows of graph g: [goff[g], goff[g+1]) (graph-major order)
};
void plan_msf(Arena &ws, const Problem &p, Msf &o);
size_t msf_scratch_bytes(const Problem &p);
dgec_status stage_msf(Ctx *c, const Problem &p, const Csr &g, const Skel &s, Msf &o, void *scratch);

// Stage D1: single-linkage dendrogram of the sorted forest.
struct Dendro {
    int32_t *a, *b;     // [E]
    int64_t *size;      // [E]
    int32_t *parent;    // [2E] parent node of every node (leaf or merge), -1 = none
    int64_t rounds = 0;
};
void plan_dendro(Arena &ws, const Problem &p, Dendro &o);
size_t dendro_scratch_bytes(const Problem &p);
dgec_status stage_dendro(Ctx *c, const Problem &p, const Csr &g, const Msf &m, Dendro &o, void *scratch);

// Stage D2: condensed tree, excess-of-mass selection and labels.
struct Condensed {
    int32_t *fall_cluster;  // [E]
    uint64_t *fall_lambda;  // [E]
    int32_t *cl_id, *cl_parent;  // [E+1]
    uint64_t *cl_birth, *cl_death, *cl_stab_hi, *cl_stab_lo;
    int64_t *cl_size;
    int32_t *cl_selected;
    int32_t *labels;  // [E]
    int32_t *gclusters;  // [G] final clusters per graph
    int64_t n_cl = 0;
    int32_t n_clusters = 0;
};
void plan_condensed(Arena &ws, const Problem &p, Condensed &o);
size_t condense_scratch_bytes(const Problem &p);
dgec_status stage_condense(Ctx *c, const Problem &p, const Msf &m, const Dendro &d, Condensed &o,
                           void *scratch);

}  // namespace dgec
