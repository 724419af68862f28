// redund.cu -- plan of the redundancy-aware expansion of V (Appendix A of
// arXiv:2312.09763); host code, no device work.
//
// Baselines (a <= b) with equal vectors b_ab = x_a - x_b and equal beams have
// equal visibilities, and a baseline whose vector is the reverse of another's
// (beams swapped) has the conjugate visibility; each such group is simulated
// once, at its representative, the first member in lexicographic order.
// Appendix A's heuristic then covers the representatives (a, b) with few
// sub-matrices V'_x = A_x B_x^dagger: the first antennas, sorted by how many
// representatives they lead, are cut into N_sub consecutive slices whose
// density (representatives / slice size) stays above a threshold tau,
// lowered step by step until the last slice also meets it; B_x holds every
// second antenna of slice x.  Here each sub-matrix becomes a block of
// contiguous rows and columns of V in a permuted antenna order (the Z planes
// are built in that order), so that the tensor-core HERK reads it with plain
// tiled loads; the order makes the slices contiguous and, for two slices,
// also the second slice's columns.  Every cover is costed in the HERK's
// 128-row tiles and the cheapest one is kept, or the whole lower triangle if
// no cover is cheaper.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "redund.h"

namespace mv {
namespace {

struct GroupKey {
    long long x, y, z;
    int b0, b1;
    bool operator==(const GroupKey& o) const {
        return x == o.x && y == o.y && z == o.z && b0 == o.b0 && b1 == o.b1;
    }
};
struct GroupKeyHash {
    size_t operator()(const GroupKey& k) const {
        unsigned long long h = 1469598103934665603ull;
        for (long long v : {k.x, k.y, k.z, (long long)k.b0, (long long)k.b1}) {
            h ^= (unsigned long long)v;
            h *= 1099511628211ull;
        }
        return (size_t)h;
    }
};

// 128-row x tile_n-column tiles of a block of nr x nc antennas (2 n_feed real
// rows per antenna).
long long block_tiles(long long nr, long long nc, int nf, int tile_n) {
    const long long rows = 2ll * nf * nr, cols = 2ll * nf * nc;
    return (rows + 127) / 128 * ((cols + tile_n - 1) / tile_n);
}

// Tiles of the whole lower triangle, as the HERK lays them out (row panels of
// 128; panel i needs the columns below its diagonal, the last chunk of a
// 256-column tiling only as wide as needed).
long long triangle_tiles(int n_ant, int nf, int tile_n) {
    const long long rows = 2ll * nf * n_ant, r16 = (rows + 15) / 16 * 16;
    long long n = 0;
    for (long long i = 0; i * 128 < rows; ++i) {
        const long long cmax = tile_n == 128 ? 128 * (i + 1) : std::min(128 * (i + 1), r16);
        n += (cmax + tile_n - 1) / tile_n;
    }
    return n;
}

struct Cover {
    int n_sub = 0;
    std::vector<int> perm;
    std::vector<RedBlock> blocks;
    long long tiles = 0;
};

// Appendix A's cuts of alpha' for n_sub slices (threshold lowered in steps of
// 0.01 from 1 until the last slice is as dense as the threshold), then the
// antenna order and blocks.
Cover sub_matrix_cover(int n_ant, const std::vector<int>& first, const std::vector<int>& second, int n_sub, int nf,
                       int tile_n) {
    std::vector<std::vector<int>> part(n_ant);
    for (size_t i = 0; i < first.size(); ++i) part[first[i]].push_back(second[i]);
    std::vector<int> ap;  // alpha': first antennas by decreasing multiplicity
    for (int a = 0; a < n_ant; ++a)
        if (!part[a].empty()) ap.push_back(a);
    std::stable_sort(ap.begin(), ap.end(), [&](int x, int y) { return part[x].size() > part[y].size(); });
    const int na = (int)ap.size();
    n_sub = std::max(1, std::min(n_sub, na));
    std::vector<char> seen(n_ant);
    // density of ap[pos, pos + n)
    auto density = [&](int pos, int n) {
        std::fill(seen.begin(), seen.end(), 0);
        long long pairs = 0, cols = 0;
        for (int i = pos; i < pos + n; ++i) {
            pairs += (long long)part[ap[i]].size();
            for (int b : part[ap[i]])
                if (!seen[b]) { seen[b] = 1; ++cols; }
        }
        return cols ? (double)pairs / ((double)n * (double)cols) : 0.0;
    };
    std::vector<int> sizes;
    for (int step = 0; step <= 100; ++step) {
        const double tau = 1.0 - 0.01 * step;
        sizes.clear();
        int pos = 0;
        for (int x = 0; x + 1 < n_sub; ++x) {
            std::fill(seen.begin(), seen.end(), 0);
            long long pairs = 0, cols = 0;
            int best = 1;
            const int max_n = na - pos - (n_sub - 1 - x);
            for (int n = 1; n <= max_n; ++n) {
                const int a = ap[pos + n - 1];
                pairs += (long long)part[a].size();
                for (int b : part[a])
                    if (!seen[b]) { seen[b] = 1; ++cols; }
                if ((double)pairs / ((double)n * (double)cols) >= tau) best = n;
                else break;
            }
            sizes.push_back(best);
            pos += best;
        }
        sizes.push_back(na - pos);
        if (density(pos, na - pos) >= tau) break;
    }
    // slices S_x, their column sets B_x, and the antennas R that lead no pair
    std::vector<int> slice_of(n_ant, -1);
    std::vector<std::vector<int>> S(n_sub);
    for (int x = 0, pos = 0; x < n_sub; pos += sizes[x], ++x)
        for (int i = pos; i < pos + sizes[x]; ++i) {
            S[x].push_back(ap[i]);
            slice_of[ap[i]] = x;
        }
    std::vector<std::vector<char>> inB(n_sub, std::vector<char>(n_ant, 0));
    for (int x = 0; x < n_sub; ++x)
        for (int a : S[x])
            for (int b : part[a]) inB[x][b] = 1;
    std::vector<int> R;
    for (int a = 0; a < n_ant; ++a)
        if (slice_of[a] < 0) R.push_back(a);
    // antenna order: slices contiguous; with two slices also the second
    // slice's columns, up to the part of slice 0 outside them
    std::vector<int> order;
    if (n_sub == 2) {
        const std::vector<char>& b1 = inB[1];
        for (int a : R) if (b1[a]) order.push_back(a);
        for (int a : S[0]) if (!b1[a]) order.push_back(a);
        for (int a : S[0]) if (b1[a]) order.push_back(a);
        for (int a : S[1]) if (b1[a]) order.push_back(a);
        for (int a : S[1]) if (!b1[a]) order.push_back(a);
        for (int a : R) if (!b1[a]) order.push_back(a);
    } else {
        for (int x = 0; x < n_sub; ++x) order.insert(order.end(), S[x].begin(), S[x].end());
        order.insert(order.end(), R.begin(), R.end());
    }
    Cover cv;
    cv.n_sub = n_sub;
    cv.perm.assign(n_ant, 0);
    for (int i = 0; i < n_ant; ++i) cv.perm[order[i]] = i;
    for (int x = 0; x < n_sub; ++x) {
        RedBlock bk{n_ant, -1, n_ant, -1};
        for (int a : S[x]) {
            bk.r0 = std::min(bk.r0, cv.perm[a]);
            bk.r1 = std::max(bk.r1, cv.perm[a] + 1);
        }
        for (int b = 0; b < n_ant; ++b)
            if (inB[x][b]) {
                bk.c0 = std::min(bk.c0, cv.perm[b]);
                bk.c1 = std::max(bk.c1, cv.perm[b] + 1);
            }
        cv.blocks.push_back(bk);
        cv.tiles += block_tiles(bk.r1 - bk.r0, bk.c1 - bk.c0, nf, tile_n);
    }
    return cv;
}

}  // namespace

bool plan_redundancy(int n_ant, const double* enu, const int* beam_idx, double tol_m, int n_feed, int tile_n,
                     RedPlan& out, const char** why) {
    *why = nullptr;
    if (n_ant < 1 || !enu) { *why = "no antennas"; return false; }
    if (!(tol_m > 0) || !std::isfinite(tol_m)) { *why = "tolerance must be positive"; return false; }
    if (n_feed < 1 || (tile_n != 128 && tile_n != 256)) { *why = "bad feed count or tile width"; return false; }
    out = RedPlan{};
    out.n_ant = n_ant;
    const long long n_bl = (long long)n_ant * (n_ant + 1) / 2;
    out.group_of.assign(n_bl, 0);
    out.conj_of.assign(n_bl, 0);
    std::unordered_map<GroupKey, int, GroupKeyHash> groups;
    groups.reserve((size_t)std::min<long long>(n_bl, 1 << 20));
    std::vector<char> rep_flip;
    long long idx = 0;
    for (int a = 0; a < n_ant; ++a)
        for (int b = a; b < n_ant; ++b, ++idx) {
            long long q[3];
            for (int k = 0; k < 3; ++k) q[k] = std::llround((enu[3 * a + k] - enu[3 * b + k]) / tol_m);
            const bool flip = q[0] < 0 || (q[0] == 0 && (q[1] < 0 || (q[1] == 0 && q[2] < 0)));
            const int ba = beam_idx ? beam_idx[a] : 0, bb = beam_idx ? beam_idx[b] : 0;
            const GroupKey key = flip ? GroupKey{-q[0], -q[1], -q[2], bb, ba} : GroupKey{q[0], q[1], q[2], ba, bb};
            auto it = groups.find(key);
            int g;
            if (it == groups.end()) {
                g = (int)out.rep_a.size();
                groups.emplace(key, g);
                out.rep_a.push_back(a);
                out.rep_b.push_back(b);
                rep_flip.push_back(flip);
            } else {
                g = it->second;
            }
            out.group_of[idx] = g;
            out.conj_of[idx] = (int8_t)(flip != (bool)rep_flip[g]);
        }
    // covers of the representatives in both orientations, 1 to 3 sub-matrices
    out.tiles_full = triangle_tiles(n_ant, n_feed, tile_n);
    out.kind = 0;
    out.n_sub = 1;
    out.tiles = out.tiles_full;
    out.perm.resize(n_ant);
    for (int a = 0; a < n_ant; ++a) out.perm[a] = a;
    out.blocks = {RedBlock{0, n_ant, 0, n_ant}};
    for (int kind = 1; kind <= 2; ++kind)
        for (int ns = 1; ns <= 3; ++ns) {
            const std::vector<int>& f = kind == 1 ? out.rep_a : out.rep_b;
            const std::vector<int>& s = kind == 1 ? out.rep_b : out.rep_a;
            Cover cv = sub_matrix_cover(n_ant, f, s, ns, n_feed, tile_n);
            if (cv.tiles < out.tiles) {
                out.kind = kind;
                out.n_sub = cv.n_sub;
                out.perm = cv.perm;
                out.blocks = cv.blocks;
                out.tiles = cv.tiles;
            }
        }
    return true;
}

}  // namespace mv
