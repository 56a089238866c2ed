// Stage L: discrete dendrogram (Alg. 5) over the skeleton, and its rows
// for condensing (Sec. 3).
#pragma once

#include "stages.cuh"

namespace dgec {

constexpr int kMaxLevels = 64;  // thresholds per run

struct Levels {
    int q = 0;
    int64_t *omega;      // [q] thresholds (device copy)
    int32_t *mlevel;     // [E] level at which x stops naming its component, -1 never
    int32_t *mparent;    // [E] the component it then joins (smallest member), -1 never
    int64_t *ncomp;      // [q] components per level
    int32_t *dense;      // [q*E] per-level labels, or null
    Msf rows;            // D's edges as forest rows (parent, x, omega), (level, x) order
    int64_t n_merges = 0;
};
void plan_levels(Arena &ws, const Problem &p, int q, bool dense, Levels &o);
size_t levels_scratch_bytes(const Problem &p);
dgec_status stage_levels(Ctx *c, const Problem &p, const Csr &g, const Skel &sk, const int64_t *h_omega,
                         Levels &o, void *scratch);
dgec_status build_level_rows(Ctx *c, const Problem &p, const Csr &g, Levels &o, void *scratch);

}  // namespace dgec
