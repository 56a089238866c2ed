// Stage H: skeleton of a dynamic hypergraph (Sec. 4.4); the forest,
// dendrogram and condense stages then run on it unchanged.
#pragma once

#include "stages.cuh"

namespace dgec {

struct HyperProblem {
    const int64_t *t;       // [E] hyperedge times
    int64_t E, V;
    const int64_t *s_off;   // [E+1] members (undirected) or sources (directed)
    const int32_t *s_vert;  // [Ms]
    int64_t Ms;
    const int64_t *d_off;   // [E+1] targets (directed only)
    const int32_t *d_vert;  // [Md]
    int64_t Md;
    bool directed;
};

// Per-vertex lists of hyperedges in (t, id) order.
struct HyperLists {
    int64_t *voff;  // [V+1]
    int32_t *id;    // [M] original hyperedge ids
    int32_t *r;     // [M] internal ids
    int64_t *tt;    // [M] times
    int32_t *vx;    // [M] vertex of each slot
};

void plan_hyper(Arena &ws, const HyperProblem &h, Csr &g, HyperLists &S, HyperLists &D, Skel &sk);
size_t hyper_scratch_bytes(const HyperProblem &h);
// Fills g.orig_of / rank_of / it, the lists, the skeleton, and p.idbits /
// tbits / tmin for the later stages.
dgec_status stage_hyper(Ctx *c, Problem &p, const HyperProblem &h, Csr &g, HyperLists &S, HyperLists &D, Skel &sk,
                        void *scratch);

}  // namespace dgec
