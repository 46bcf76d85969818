// Partition trees of the k-input multiplier (Section V-C, Table II).
//
// Notation: "(4,3)|(2,2)" -- layers separated by '|', the group list of a
// layer splits, left to right, the next not-yet-split group of the layer
// above whose size equals the list's sum. A group of size g >= 2 that is
// never split multiplies g inputs directly; a group of size 1 is an input.
//
// A node with m children rescales m - 1 times (Algorithm 1) unless it is the
// root, whose m - 1 rescales follow the relinearisation. Depth = the largest
// sum of rescales on a leaf-to-root path; valid iff depth <= ceil(log2 k).
#include "plan.h"

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstring>

namespace ckks {

static const char *kTableII[13] = {
    nullptr, nullptr, "(1,1)", "(1,1,1)", "(2,2)", "(2,2,1)", "(3,3)", "(4,3)|(2,2)", "(4,4)|(2,2),(2,2)",
    "(3,3,3)", "(3,3,4)|(2,2)", "(4,4,3)|(2,2),(2,2)", "(6,6)|(3,3),(3,3)"};

const char *table_ii_partition(int k) { return (k >= 2 && k <= 12) ? kTableII[k] : nullptr; }

// parse "(a,b,...),(c,...)" into group lists
static bool parse_layer(const std::string &s, std::vector<std::vector<int>> &out) {
    size_t i = 0;
    while (i < s.size()) {
        if (s[i] == ',' || isspace((unsigned char)s[i])) { ++i; continue; }
        if (s[i] != '(') return false;
        ++i;
        std::vector<int> g;
        while (i < s.size() && s[i] != ')') {
            if (s[i] == ',' || isspace((unsigned char)s[i])) { ++i; continue; }
            if (!isdigit((unsigned char)s[i])) return false;
            int v = 0;
            while (i < s.size() && isdigit((unsigned char)s[i])) { v = v * 10 + (s[i] - '0'); ++i; if (v > 64) return false; }
            if (v < 1) return false;
            g.push_back(v);
        }
        if (i >= s.size()) return false;
        ++i;  // ')'
        if (g.empty()) return false;
        out.push_back(g);
    }
    return !out.empty();
}

static int ceil_log2(int k) {
    int d = 0;
    while ((1 << d) < k) ++d;
    return d;
}

int plan_build(Plan &P, int k, const char *partition) {
    if (k < 2 || k > 12) return -1;
    std::string text = partition ? partition : table_ii_partition(k);
    std::vector<std::vector<std::vector<int>>> layers;
    size_t start = 0;
    while (true) {
        size_t bar = text.find('|', start);
        std::string part = text.substr(start, bar == std::string::npos ? std::string::npos : bar - start);
        std::vector<std::vector<int>> groups;
        if (!parse_layer(part, groups)) return -1;
        layers.push_back(groups);
        if (bar == std::string::npos) break;
        start = bar + 1;
    }
    if (layers[0].size() != 1) return -1;
    // build nodes: tmp tree with sizes
    struct T {
        int size;
        std::vector<int> kids;
    };
    std::vector<T> t;
    t.push_back({k, {}});
    int sum = 0;
    for (int g : layers[0][0]) sum += g;
    if (sum != k || layers[0][0].size() < 2) return -1;
    std::vector<int> frontier;
    for (int g : layers[0][0]) {
        t.push_back({g, {}});
        t[0].kids.push_back((int)t.size() - 1);
        frontier.push_back((int)t.size() - 1);
    }
    for (size_t li = 1; li < layers.size(); ++li) {
        std::vector<int> next;
        std::vector<bool> used(frontier.size(), false);
        for (auto &grp : layers[li]) {
            int s = 0;
            for (int g : grp) s += g;
            if (grp.size() < 2) return -1;
            bool placed = false;
            for (size_t fi = 0; fi < frontier.size(); ++fi) {
                if (!used[fi] && t[frontier[fi]].size == s) {
                    used[fi] = true;
                    for (int g : grp) {
                        t.push_back({g, {}});
                        t[frontier[fi]].kids.push_back((int)t.size() - 1);
                        next.push_back((int)t.size() - 1);
                    }
                    placed = true;
                    break;
                }
            }
            if (!placed) return -1;
        }
        frontier = next;
    }
    // undivided groups of size >= 2 multiply that many leaves
    for (size_t i = 0; i < t.size(); ++i) {
        if (t[i].size >= 2 && t[i].kids.empty()) {
            for (int j = 0; j < t[i].size; ++j) {
                t.push_back({1, {}});
                t[i].kids.push_back((int)t.size() - 1);
            }
        }
    }
    // post-order into plan nodes; leaves numbered left to right
    P = Plan();
    P.k = k;
    P.text = text;
    int leaf = 0;
    std::vector<int> map(t.size(), -1);
    // iterative post-order
    std::vector<std::pair<int, size_t>> st;
    st.push_back({0, 0});
    while (!st.empty()) {
        auto &top = st.back();
        int id = top.first;
        if (t[id].size == 1 && t[id].kids.empty()) {
            map[id] = -1 - leaf;  // negative: leaf index
            ++leaf;
            st.pop_back();
            continue;
        }
        if (top.second < t[id].kids.size()) {
            int kid = t[id].kids[top.second++];
            st.push_back({kid, 0});
            continue;
        }
        PlanNode n;
        n.size = t[id].size;
        for (int kid : t[id].kids) n.children.push_back(map[kid]);
        n.mu = (int)t[id].kids.size() - 1;
        n.root = id == 0;
        P.nodes.push_back(n);
        map[id] = (int)P.nodes.size() - 1;
        st.pop_back();
    }
    if (leaf != k) return -1;
    // depth, rescale units
    std::vector<int> depth(P.nodes.size(), 0);
    P.rs_units = 0;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        int dmax = 0;
        for (int c : P.nodes[i].children)
            if (c >= 0 && depth[c] > dmax) dmax = depth[c];
        depth[i] = P.nodes[i].mu + dmax;
        if (!P.nodes[i].root) P.rs_units += P.nodes[i].size + 1;
    }
    P.depth = depth.back();
    if (P.depth > ceil_log2(k)) return -2;
    return 0;
}

// Levels at each node for an input level; polys of each node's output.
void plan_levels(const Plan &P, int level, std::vector<int> &lvl_in, std::vector<int> &lvl_out,
                 std::vector<int> &polys) {
    size_t n = P.nodes.size();
    lvl_in.assign(n, 0);
    lvl_out.assign(n, 0);
    polys.assign(n, 0);
    for (size_t i = 0; i < n; ++i) {
        int lmin = 1 << 30, p = 1;
        for (int c : P.nodes[i].children) {
            int cl = c >= 0 ? lvl_out[c] : level;
            int cp = c >= 0 ? polys[c] : 2;
            if (cl < lmin) lmin = cl;
            p += cp - 1;
        }
        lvl_in[i] = lmin;
        lvl_out[i] = lmin - P.nodes[i].mu;
        polys[i] = P.nodes[i].root ? 2 : p;
    }
}

}  // namespace ckks

namespace ckks {

// ---------------------------------------------------------------------------
// Partition search (Section V-C asks for the partition of lowest complexity
// among those that keep the depth at ceil(log2 k)). Every valid tree is
// enumerated; each is costed by one criterion:
//   kCostRsUnits   Table II's count: size + 1 rescale units per non-root node;
//   kCostTransforms limb (I)NTTs of the whole k-input multiply at an input
//                  level (Algorithm 1 at inner nodes: level per polynomial;
//                  the root's relinearisation and relocated rescale).
// The text of the cheapest tree in the layered notation is parsed back and
// re-costed, so the returned partition is exactly the tree that was costed.
// ---------------------------------------------------------------------------
namespace {

struct TNode {
    int size;
    std::vector<TNode> kids;  // empty: a leaf (size 1) or an undivided group
    int depth() const {
        if (kids.empty()) return size >= 2 ? size - 1 : 0;
        int d = 0;
        for (auto &k : kids) d = std::max(d, k.depth());
        return (int)kids.size() - 1 + d;
    }
};

// all sub-trees over g inputs with depth <= budget
void subtrees(int g, int budget, std::vector<TNode> &out);

void split_into(int remaining, int maxpart, std::vector<int> &parts, std::vector<std::vector<int>> &all) {
    if (remaining == 0) {
        all.push_back(parts);
        return;
    }
    for (int p = std::min(remaining, maxpart); p >= 1; --p) {
        parts.push_back(p);
        split_into(remaining - p, p, parts, all);
        parts.pop_back();
    }
}

void combine(const std::vector<int> &parts, size_t i, int budget, std::vector<TNode> &cur, std::vector<TNode> &out,
             int g) {
    if (i == parts.size()) {
        TNode n{g, cur};
        out.push_back(n);
        return;
    }
    std::vector<TNode> opts;
    subtrees(parts[i], budget, opts);
    for (auto &o : opts) {
        cur.push_back(o);
        combine(parts, i + 1, budget, cur, out, g);
        cur.pop_back();
    }
}

void subtrees(int g, int budget, std::vector<TNode> &out) {
    if (g == 1) {
        out.push_back(TNode{1, {}});
        return;
    }
    if (g - 1 <= budget) out.push_back(TNode{g, {}});  // undivided: g inputs, g - 1 rescales
    std::vector<std::vector<int>> all;
    std::vector<int> parts;
    split_into(g, g, parts, all);
    for (auto &ps : all) {
        const int m = (int)ps.size();
        if (m < 2 || m - 1 > budget) continue;
        bool all_ones = true;
        for (int p : ps) all_ones = all_ones && p == 1;
        if (all_ones) continue;  // same tree as the undivided group
        std::vector<TNode> cur;
        combine(ps, 0, budget - (m - 1), cur, out, g);
    }
}

// layered text; children ordered by size (desc), divided before undivided
std::string layered_text(const TNode &root) {
    std::string text;
    std::vector<const TNode *> layer{&root};
    bool first = true;
    while (!layer.empty()) {
        std::vector<const TNode *> next;
        std::string groups;
        for (const TNode *n : layer) {
            if (n->kids.empty()) continue;
            std::vector<const TNode *> kids;
            for (auto &k : n->kids) kids.push_back(&k);
            std::stable_sort(kids.begin(), kids.end(), [](const TNode *a, const TNode *b) {
                if (a->size != b->size) return a->size > b->size;
                return !a->kids.empty() && b->kids.empty();
            });
            groups += "(";
            for (size_t i = 0; i < kids.size(); ++i) groups += (i ? "," : "") + std::to_string(kids[i]->size);
            groups += "),";
            for (auto *k : kids) next.push_back(k);
        }
        if (groups.empty()) break;
        groups.pop_back();
        text += (first ? "" : "|") + groups;
        first = false;
        layer = next;
    }
    return text;
}

}  // namespace

double plan_cost(const Plan &P, int criterion, int level, int K, int alpha) {
    if (criterion == kCostRsUnits) return P.rs_units;
    if (criterion == kCostPrecision) {
        // the largest degree (inputs below the node) of a tuple rescaled
        // before relinearisation, then limb transforms as the tie-break
        int deg = 0;
        for (const PlanNode &n : P.nodes)
            if (!n.root) deg = std::max(deg, n.size);
        return 1e6 * deg + plan_cost(P, kCostTransforms, level, K, alpha);
    }
    std::vector<int> lin, lout, polys;
    plan_levels(P, level, lin, lout, polys);
    double c = 0;
    for (size_t i = 0; i < P.nodes.size(); ++i) {
        const PlanNode &n = P.nodes[i];
        if (!n.root) {
            c += (double)(n.size + 1) * lin[i];  // Algorithm 1: l transforms per polynomial
        } else {
            const int l = lin[i], nn = P.k, mu = n.mu;
            const int digits = (l + alpha - 1) / alpha;
            double modup = 0;
            for (int b = 0; b < digits; ++b) modup += l + K - std::min(alpha, l - b * alpha);
            c += (nn - 1) * l + (nn - 1) * modup + 2.0 * K + 2.0 * l + 2.0 * (l - mu);
        }
    }
    return c;
}

int plan_optimize(int k, int criterion, int level, int K, int alpha, std::string &best_text, double &best_cost) {
    if (k < 2 || k > 12) return -1;
    const int D = ceil_log2(k);
    if ((criterion == kCostTransforms || criterion == kCostPrecision) && level <= D) return -2;
    std::vector<TNode> roots;
    std::vector<std::vector<int>> all;
    std::vector<int> parts;
    split_into(k, k, parts, all);
    for (auto &ps : all) {
        const int m = (int)ps.size();
        if (m < 2 || m - 1 > D) continue;
        std::vector<TNode> cur;
        combine(ps, 0, D - (m - 1), cur, roots, k);
    }
    best_cost = 1e300;
    best_text.clear();
    size_t best_nodes = 0;
    for (auto &r : roots) {
        std::string t = layered_text(r);
        Plan P;
        if (plan_build(P, k, t.c_str()) != 0) continue;  // the text must parse back to a valid tree
        double c = plan_cost(P, criterion, level, K, alpha);
        const bool better = c < best_cost - 1e-9 ||
                            (std::fabs(c - best_cost) < 1e-9 &&
                             (P.nodes.size() < best_nodes || (P.nodes.size() == best_nodes && t < best_text)));
        if (better) {
            best_cost = c;
            best_text = t;
            best_nodes = P.nodes.size();
        }
    }
    return best_text.empty() ? -1 : 0;
}

}  // namespace ckks
