// redund.h -- plan of the redundancy-aware expansion of V (Appendix A of
// arXiv:2312.09763, "Utilising baseline redundancies"); host code.
#pragma once
#include <cstdint>
#include <vector>

namespace mv {

// A block of the expansion: rows [r0, r1) x columns [c0, c1) of V in the
// plan's antenna order (antenna a sits at position perm[a]).
struct RedBlock {
    int r0, r1, c0, c1;
};

struct RedPlan {
    int n_ant = 0;
    // redundant groups of the baselines (a <= b): one representative pair
    // each, the first member in lexicographic order
    std::vector<int> rep_a, rep_b;
    // per baseline (a <= b, row-major over a then b): its group, and whether
    // it is a reversed baseline of the group (V_ab^{pq} = conj(V_rep^{qp}))
    std::vector<int> group_of;
    std::vector<int8_t> conj_of;
    // the cover: kind 0 = the whole lower triangle (no sub-matrices), 1 =
    // sub-matrices of the representatives as (row a, column b), 2 = as (row b,
    // column a); perm and blocks place them; n_sub sub-matrices
    int kind = 0, n_sub = 1;
    std::vector<int> perm;
    std::vector<RedBlock> blocks;
    long long tiles = 0;       // cost of the cover in tensor-core tiles
    long long tiles_full = 0;  // the same for the whole lower triangle
};

// Groups the baselines of n_ant antennas (ENU metres [n_ant][3], beam index
// per antenna) whose vectors agree to tol_m (rounded to a tol_m grid) and
// whose beams agree; a baseline and the reverse of another are one group
// (V_ba = conj(V_ab)).  Then the sub-matrix heuristic of Appendix A on the
// representatives, in both orientations and for 1 to 3 sub-matrices, each
// cover costed in 128-row x tile_n-column tiles of the 2 n_feed-row real
// Gram matrix; the cheapest cover, or the whole triangle if nothing is
// cheaper, is returned.  False (with a message) on bad input.
bool plan_redundancy(int n_ant, const double* enu, const int* beam_idx, double tol_m, int n_feed, int tile_n,
                     RedPlan& out, const char** why);

}  // namespace mv
