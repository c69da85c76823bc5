// catalog.cpp -- treelet shapes (Section 3.2.1) and the per-k index programs
// of the table build (Eq. 1).  Host code, computed once per process.
#include "catalog.h"

#include <algorithm>
#include <map>
#include <mutex>

namespace mc {

int binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int colex_rank(unsigned mask)
{
    int r = 0, i = 0;
    for (int p = 0; mask; ++p, mask >>= 1)
        if (mask & 1u) r += binom(p, ++i);
    return r;
}

unsigned colex_unrank(int size, int rank)
{
    unsigned mask = 0;
    for (int i = size; i >= 1; --i) {
        int p = i - 1;
        while (binom(p + 1, i) <= rank) ++p;
        rank -= binom(p, i);
        mask |= 1u << p;
    }
    return mask;
}

namespace {

// Rooted trees as strings.  A root's children are a non-increasing
// sequence of "blocks" 1 + child + 0; all such sequences with m nodes in
// total are generated directly, so every tree appears exactly once.
std::vector<std::string> trees_of_size(int h);

void forests(int m, const std::string *bound, std::string prefix, std::vector<std::string> &out)
{
    if (m == 0) { out.push_back(prefix); return; }
    for (int s = 1; s <= m; ++s)
        for (const std::string &t : trees_of_size(s)) {
            std::string block = "1" + t + "0";
            if (bound && block > *bound) continue;
            forests(m - s, &block, prefix + block, out);
        }
}

std::vector<std::string> trees_of_size(int h)
{
    static std::map<int, std::vector<std::string>> memo;
    auto it = memo.find(h);
    if (it != memo.end()) return it->second;
    std::vector<std::string> out;
    forests(h - 1, nullptr, "", out);
    std::sort(out.begin(), out.end(), [](const std::string &a, const std::string &b) {
        return std::stoull("0" + a, nullptr, 2) < std::stoull("0" + b, nullptr, 2);
    });
    memo[h] = out;
    return out;
}

std::vector<std::string> blocks_of(const std::string &s)
{
    std::vector<std::string> out;
    int depth = 0;
    size_t start = 0;
    for (size_t i = 0; i < s.size(); ++i) {
        depth += s[i] == '1' ? 1 : -1;
        if (depth == 0) { out.push_back(s.substr(start, i + 1 - start)); start = i + 1; }
    }
    return out;
}

// adjacency of the tree drawn by s (node 0 = root, DFS numbering)
std::vector<std::vector<int>> tree_adjacency(const std::string &s)
{
    std::vector<std::vector<int>> adj(1);
    std::vector<int> path{0};
    for (char ch : s) {
        if (ch == '1') {
            int x = (int)adj.size();
            adj.emplace_back();
            adj[path.back()].push_back(x);
            adj[x].push_back(path.back());
            path.push_back(x);
        } else {
            path.pop_back();
        }
    }
    return adj;
}

std::string rooted_string(const std::vector<std::vector<int>> &adj, int v, int parent)
{
    std::vector<std::string> kids;
    for (int u : adj[v])
        if (u != parent) kids.push_back("1" + rooted_string(adj, u, v) + "0");
    std::sort(kids.begin(), kids.end(), std::greater<std::string>());
    std::string s;
    for (auto &x : kids) s += x;
    return s;
}

uint32_t to_code(const std::string &s)
{
    uint32_t c = 0;
    for (char ch : s) c = (c << 1) | (ch == '1');
    return c;
}

}  // namespace

const ShapeCatalog &shape_catalog()
{
    static ShapeCatalog cat;
    static std::once_flag once;
    std::call_once(once, [] {
        std::map<std::pair<int, std::string>, int> gid;
        for (int h = 1; h <= MAXK; ++h) {
            cat.first[h] = (int)cat.shapes.size();
            std::vector<std::string> ts = trees_of_size(h);
            cat.r[h] = (int)ts.size();
            // unrooted code: the smallest s_T over all rootings
            std::vector<uint32_t> ucodes;
            std::vector<uint32_t> per_shape;
            for (auto &s : ts) {
                auto adj = tree_adjacency(s);
                uint32_t best = 0xffffffffu;
                for (int v = 0; v < (int)adj.size(); ++v)
                    best = std::min(best, to_code(rooted_string(adj, v, -1)));
                per_shape.push_back(best);
                ucodes.push_back(best);
            }
            std::sort(ucodes.begin(), ucodes.end());
            ucodes.erase(std::unique(ucodes.begin(), ucodes.end()), ucodes.end());
            cat.n_unrooted[h] = (int)ucodes.size();
            for (int i = 0; i < (int)ts.size(); ++i) {
                Shape sh;
                sh.str = ts[i];
                sh.code = to_code(ts[i]);
                sh.size = h;
                sh.local = i;
                sh.unrooted = (int)(std::lower_bound(ucodes.begin(), ucodes.end(), per_shape[i]) -
                                    ucodes.begin());
                if (h > 1) {
                    auto bl = blocks_of(ts[i]);
                    std::string right = bl[0].substr(1, bl[0].size() - 2);
                    std::string left;
                    for (size_t j = 1; j < bl.size(); ++j) left += bl[j];
                    sh.beta = (int)std::count(bl.begin(), bl.end(), bl[0]);
                    sh.left = gid.at({(int)left.size() / 2 + 1, left});
                    sh.right = gid.at({(int)right.size() / 2 + 1, right});
                }
                gid[{h, ts[i]}] = (int)cat.shapes.size();
                cat.shapes.push_back(sh);
            }
        }
        cat.first[MAXK + 1] = (int)cat.shapes.size();
    });
    return cat;
}

Geometry make_geometry(int k)
{
    const ShapeCatalog &cat = shape_catalog();
    Geometry g;
    g.k = k;
    for (int h = 1; h <= k; ++h) {
        g.Bc[h] = binom(k - 1, h - 1);
        g.Bs[h] = binom(k - 1, h);
        g.Wc[h] = cat.r[h] * g.Bc[h];
        g.Ws[h] = cat.r[h] * g.Bs[h];
    }
    return g;
}

static int shape_gid(const ShapeCatalog &cat, const std::string &str)
{
    const int h = (int)str.size() / 2 + 1;
    for (int i = 0; i < cat.r[h]; ++i)
        if (cat.shapes[cat.gid(h, i)].str == str) return cat.gid(h, i);
    return -1;
}

// balanced decomposition of a rooted k-shape: false when none exists
static bool balanced(const ShapeCatalog &cat, const std::string &str, int k, int &left, int &right, int &beta)
{
    const std::vector<std::string> bl = blocks_of(str);
    for (size_t i = 0; i < bl.size(); ++i) {
        const int sz = (int)bl[i].size() / 2;
        if (sz < 2 || sz > k - 2) continue;
        std::string rest;
        for (size_t j = 0; j < bl.size(); ++j)
            if (j != i) rest += bl[j];
        left = shape_gid(cat, rest);
        right = shape_gid(cat, bl[i].substr(1, bl[i].size() - 2));
        beta = (int)std::count(bl.begin(), bl.end(), bl[i]);
        return true;
    }
    return false;
}

static Programs build_programs(int k, bool skip)
{
    const ShapeCatalog &cat = shape_catalog();
    Programs P;
    P.geo = make_geometry(k);
    P.skip = skip;
    const Geometry &G = P.geo;
    for (int i = 0; i < MAX_SHAPES; ++i) P.bal_left[i] = P.bal_right[i] = -1, P.bal_beta[i] = 1;
    for (int j = 0; j < 32; ++j) P.copies[j] = k;
    if (skip) {
        for (int s = 0; s < cat.r[k]; ++s) {
            const int g = cat.gid(k, s);
            int l, r, b;
            if (balanced(cat, cat.shapes[g].str, k, l, r, b)) P.bal_left[g] = l, P.bal_right[g] = r, P.bal_beta[g] = b;
        }
        // a_j: nodes of tree j at which its rooting has a balanced decomposition
        for (int j = 0; j < cat.n_unrooted[k]; ++j) {
            int rep = -1;
            for (int s = 0; s < cat.r[k] && rep < 0; ++s)
                if (cat.shapes[cat.gid(k, s)].unrooted == j) rep = cat.gid(k, s);
            const auto adj = tree_adjacency(cat.shapes[rep].str);
            int a = 0;
            for (int x = 0; x < (int)adj.size(); ++x) {
                int l, r, b;
                a += balanced(cat, rooted_string(adj, x, -1), k, l, r, b) ? 1 : 0;
            }
            P.copies[j] = a;
        }
    }
    // outputs in row order: set-major, o = rho * r_h + s (every shape of
    // one colour set side by side)
    for (int h = 2; h <= k; ++h) {
        if (skip && h == k - 1) continue;
        MergeLevel &M = P.merge[h];
        for (int rho = 0; rho < G.Bc[h]; ++rho) {
            // D: the h-1 colours of C other than c_v, as a relative set
            const unsigned D = colex_unrank(h - 1, rho);
            for (int s = 0; s < cat.r[h]; ++s) {
                const Shape &T = cat.shapes[cat.gid(h, s)];
                int left = T.left, right = T.right, beta = T.beta;
                if (skip && h == k) {
                    left = P.bal_left[cat.gid(h, s)], right = P.bal_right[cat.gid(h, s)], beta = P.bal_beta[cat.gid(h, s)];
                    if (left < 0) {  // not counted: no terms
                        M.offset.push_back((int32_t)M.terms.size());
                        M.info.push_back(1 | (1 << 4) | (1 << 8));
                        continue;
                    }
                }
                const Shape &A = cat.shapes[left];
                const Shape &B = cat.shapes[right];
                const int h1 = A.size, h2 = B.size;
                M.offset.push_back((int32_t)M.terms.size());
                int nterms = 0;
                for (unsigned sub = D;; sub = (sub - 1) & D) {  // D'' subset of D
                    if (__builtin_popcount(sub) == h2) {
                        const unsigned Dp = D & ~sub;        // D' = D \ D''
                        const int ia = h1 == 1 ? 0 : colex_rank(Dp) * cat.r[h1] + A.local;
                        const int ib = colex_rank(sub) * cat.r[h2] + B.local;
                        M.terms.push_back((uint32_t)ia | ((uint32_t)ib << 16));
                        ++nterms;
                    }
                    if (sub == 0) break;
                }
                M.info.push_back(h1 | (h2 << 4) | (beta << 8) | (nterms << 16));
            }
        }
    }
    for (int h = 1; h <= k - 1; ++h) {
        if (skip && h == k - 1) continue;
        GatherLevel &L = P.gather[h];
        L.map.assign((size_t)k * k * G.Bs[h], -1);
        for (int cv = 0; cv < k; ++cv)
            for (int cu = 0; cu < k; ++cu) {
                if (cu == cv) continue;
                for (int rho = 0; rho < G.Bs[h]; ++rho) {
                    // absolute colour set C'' of S entry rho at a node of colour cv
                    unsigned rel = colex_unrank(h, rho);
                    unsigned C2 = (rel & ((1u << cv) - 1u)) | ((rel >> cv) << (cv + 1));
                    if (!(C2 >> cu & 1u)) continue;
                    unsigned rest = C2 & ~(1u << cu);
                    unsigned relu = (rest & ((1u << cu) - 1u)) | ((rest >> (cu + 1)) << cu);
                    L.map[((size_t)cv * k + cu) * G.Bs[h] + rho] = (int16_t)colex_rank(relu);
                }
            }
    }
    return P;
}

const Programs &programs(int k, bool skip)
{
    static Programs cache[2][MAXK + 1];
    static std::once_flag once[2][MAXK + 1];
    std::call_once(once[skip][k], [k, skip] { cache[skip][k] = build_programs(k, skip); });
    return cache[skip][k];
}

}  // namespace mc
