// catalog.h -- treelet shapes and the per-k programs of the table build.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace mc {

constexpr int MAXK = 8;
constexpr int MAX_SHAPES = 200;  // rooted shapes on 1..8 nodes: 200

// One rooted treelet shape (Section 3.2.1).  `str` is s_T: a DFS from the
// root writing 1 when moving away from the root and 0 when moving back, the
// children of each node visited in decreasing lexicographic order of their
// own strings.  T'' is the subtree of the first child, T' the rest, beta the
// number of root children whose subtree equals T''.
struct Shape {
    std::string str;
    uint32_t code = 0;   // s_T as a 2(h-1)-bit integer
    int size = 0;
    int local = 0;       // rank of code among shapes of this size
    int left = -1;       // global id of T'
    int right = -1;      // global id of T''
    int beta = 1;
    int unrooted = 0;    // id of the unrooted shape within this size
};

struct ShapeCatalog {
    std::vector<Shape> shapes;  // global ids: sizes 1..8, id order within a size
    int first[MAXK + 2] = {0};
    int r[MAXK + 1] = {0};
    int n_unrooted[MAXK + 1] = {0};
    int gid(int h, int local) const { return first[h] + local; }
};

const ShapeCatalog &shape_catalog();

int binom(int n, int k);
int colex_rank(unsigned mask);       // rank among masks of the same popcount
unsigned colex_unrank(int size, int rank);  // inverse (masks over any width)

// Table geometry for k colours: row widths per level.
struct Geometry {
    int k = 0;
    int Bc[MAXK + 1] = {0};  // C(k-1, h-1): colour sets per shape in a c row
    int Bs[MAXK + 1] = {0};  // C(k-1, h): colour sets per shape in an S row
    int Wc[MAXK + 1] = {0};  // r_h * Bc[h]
    int Ws[MAXK + 1] = {0};  // r_h * Bs[h]
};
Geometry make_geometry(int k);

// Rows are set-major: entry (colour set rho, shape s) of a level-h row sits
// at rho * r_h + s, so the entries of one colour set are contiguous.
// Merge program of level h: for output entry o = rho * r_h + s the list of
// (index into the c_{|T'|} row, index into the S_{|T''|} row) pairs of
// Eq. (1), one per split of the colour set.
struct MergeLevel {
    std::vector<int32_t> info;    // per output: h1 | h2 << 4 | beta << 8 | nterms << 16
    std::vector<int32_t> offset;  // per output: first term
    std::vector<uint32_t> terms;  // ia | ib << 16
};

// Gather map of level h: S_h(v)[rho'', s] accumulates c_h(u)[src, s] over
// neighbours u and every shape s, src = map[(c_v * k + c_u) * Bs[h] + rho'']
// (-1: no contribution because c_u is not in the set).
struct GatherLevel {
    std::vector<int16_t> map;
};

// With round skipping (Section 3.3.2) level k is built from a balanced
// decomposition: T'' is the subtree of the first root child (in s_T order)
// with 2..k-2 nodes, T' the rest, beta the number of root children equal
// to T''; level k-1 is never built.  Rooted k-shapes without such a child
// (star and leaf rootings) are not counted: their merge has no terms.
struct Programs {
    Geometry geo;
    MergeLevel merge[MAXK + 1];
    GatherLevel gather[MAXK + 1];
    bool skip = false;
    int bal_left[MAX_SHAPES], bal_right[MAX_SHAPES], bal_beta[MAX_SHAPES];  // per level-k shape (global
                                                                             // ids; -1: not counted)
    int copies[32];  // per unrooted k-shape: rooted copies the level-k table holds per copy
                     // (k, or with skipping a_j, the balanced rootings; 0 for the star)
};
const Programs &programs(int k, bool skip = false);

}  // namespace mc
